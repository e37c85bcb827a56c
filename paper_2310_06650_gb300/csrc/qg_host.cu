// Host side of libqg: input validation, set-up of the network data, the dense
// reduced-Laplacian inverse and the line-outage block, descriptor tables for
// the kernels, and the C ABI declared in include/qg.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "qg_internal.h"
#include "qg_sparse.h"

using namespace qg;

namespace {

thread_local std::string g_create_error;

constexpr int BLK = 256;
constexpr int DENSE_MAX_N = 8192;  // dense Yhat^-1 is n^2 doubles

struct HostInst {
  // copies of the caller's arrays (double / int)
  int n, M, G, Z, T, K, ref;
  std::vector<int> from, to, gen_bus, gen_zone, ctg;
  std::vector<double> r, x, bch, smax, sctg, ca, cb, cr, pmin, pmax, qmin, qmax, ramp, vmin, vmax;
  std::vector<double> dt, load_p, load_q, rreq;
  // derived
  std::vector<double> y, gsr, bsr;
  std::vector<double> zinv;  // n x n, ref row/col zero
  std::vector<double> z1;    // n
  std::vector<double> lodf;  // M x K
};

}  // namespace

struct qg_ctx {
  int n_inst = 0;
  qg_options opt{};
  std::vector<HostInst> hi;
  std::vector<Inst> inst;
  long long n_x = 0;
  int maxT = 0;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  Dev<double, double> d64{};
  Dev<float, df32> d32{};
  Launch L{};
  double *d_obj = nullptr, *d_terms = nullptr;
  void *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
  void *d_xs = nullptr;     // staging for qg_eval_grad_host (Real)
  double *d_xd = nullptr;   // staging doubles (mixed mode conversions)
  long long *d_step = nullptr;
  // cached CUDA graph of one (eval + Adam) iteration for qg_solve
  cudaGraphExec_t gexec = nullptr;
  const void *g_x = nullptr;
  double g_lr = 0, g_b1 = 0, g_b2 = 0;
  double *g_trace = nullptr;
  // optional per-kernel timing: ev[0..9] bracket the nine evaluation kernels, ev[10] ends Adam
  bool profiling = false;
  cudaEvent_t ev[N_PHASES + 1] = {};
  std::string err;
};

namespace {

int fail(qg_ctx *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  g_create_error = msg;
  return code;
}

#define CUDA_TRY(h, call)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail((h), QG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dalloc(qg_ctx *h, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(*p);
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
  for (auto *v : {&I.r, &I.x, &I.bch, &I.smax, &I.sctg, &I.ca, &I.cb, &I.cr, &I.pmin, &I.pmax, &I.qmin, &I.qmax,
                  &I.ramp, &I.vmin, &I.vmax, &I.dt, &I.load_p, &I.load_q, &I.rreq})
    if (!finite_all(*v)) return bad("non-finite input");
  return QG_OK;
}

// DC network set-up (Sec. II-E): y_j = -b_sr = x / (r^2 + x^2); reduced Laplacian with the
// reference bus removed; Yhat^-1 columns by sparse LDL^T solves; line-outage block
//   L[m,k] = y_m (u_k[f_m] - u_k[o_m]) / (1 - y_k (u_k[f_k] - u_k[o_k])),  u_k = Yhat^-1 a_k,
// which is the rank-1 SMW correction of Eq. rank_correct expressed on branch flows.
int build_dc(qg_ctx *h, HostInst &I, int b) {
  const int n = I.n, M = I.M, K = I.K;
  I.y.resize(M); I.gsr.resize(M); I.bsr.resize(M);
  for (int j = 0; j < M; ++j) {
    const double den = I.r[j] * I.r[j] + I.x[j] * I.x[j];
    I.y[j] = I.x[j] / den;
    I.gsr[j] = I.r[j] / den;
    I.bsr[j] = -I.x[j] / den;
  }
  // reduced index: bus i -> i' (ref removed)
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
  SparseLDL F;
  if (!F.factor(nr, off, diag))
    return fail(h, QG_ERR_ISLANDING, "instance " + std::to_string(b) + ": the DC Laplacian is singular (disconnected grid)");
  if (n > DENSE_MAX_N)
    return fail(h, QG_ERR_UNSUPPORTED, "instance " + std::to_string(b) + ": n = " + std::to_string(n) +
                                           " exceeds the dense-inverse limit " + std::to_string(DENSE_MAX_N));
  // dense inverse (n x n, zero ref row and column), columns by solves
  I.zinv.assign((size_t)n * n, 0.0);
  std::vector<double> col(nr);
  for (int cc = 0; cc < nr; ++cc) {
    std::fill(col.begin(), col.end(), 0.0);
    col[cc] = 1.0;
    F.solve(col.data());
    // bus id of reduced column cc
    const int bc = cc < I.ref ? cc : cc + 1;
    for (int rr = 0; rr < nr; ++rr) {
      const int br = rr < I.ref ? rr : rr + 1;
      I.zinv[(size_t)br * n + bc] = col[rr];
    }
  }
  // symmetrize (the two triangles agree to rounding; keep one value for bitwise symmetry)
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double v = 0.5 * (I.zinv[(size_t)i * n + j] + I.zinv[(size_t)j * n + i]);
      I.zinv[(size_t)i * n + j] = v;
      I.zinv[(size_t)j * n + i] = v;
    }
  I.z1.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += I.zinv[(size_t)i * n + j];
    I.z1[i] = s;
  }
  // line-outage block
  I.lodf.assign((size_t)M * K, 0.0);
  std::vector<int> bad_k;
  for (int k = 0; k < K; ++k) {
    const int jk = I.ctg[k];
    // u_k = Z (e_f - e_o), read from the dense inverse
    const int fk = I.from[jk], ok = I.to[jk];
    auto u = [&](int bus) { return I.zinv[(size_t)bus * n + fk] - I.zinv[(size_t)bus * n + ok]; };
    const double ptdf_kk = I.y[jk] * (u(fk) - u(ok));
    const double den = 1.0 - ptdf_kk;
    if (std::fabs(den) < 1e-9) {
      bad_k.push_back(jk);
      continue;
    }
    for (int m = 0; m < M; ++m) I.lodf[(size_t)m * K + k] = I.y[m] * (u(I.from[m]) - u(I.to[m])) / den;
  }
  if (!bad_k.empty()) {
    std::string s = "instance " + std::to_string(b) + ": outage of branch(es)";
    for (size_t q = 0; q < bad_k.size() && q < 8; ++q) s += " " + std::to_string(bad_k[q]);
    s += " islands the grid (|1 - PTDF_kk| < 1e-9)";
    return fail(h, QG_ERR_ISLANDING, s);
  }
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

// Build every device array of one precision flavour.
template <typename Real, typename Dc>
int build_device(qg_ctx *h, Dev<Real, Dc> &d) {
  const int B = h->n_inst;
  std::vector<Inst> &inst = h->inst;
  // global arrays
  std::vector<int> br_from, br_to, br_kidx, gen_bus, gen_zone, inc_ptr{0}, inc, bgen_ptr{0}, bgen, zgen_ptr{0}, zgen, ctg_br;
  std::vector<double> br_g, br_b, br_bc, br_smax, br_sctg, br_y, ga, gb, gcr, gpmax, gramp, load_p, load_q, rreq, dt, lo, hi;
  std::vector<double> zinv, z1;
  std::vector<double> lodf;
  for (int b = 0; b < B; ++b) {
    const HostInst &I = h->hi[b];
    const Inst &D = inst[b];
    for (int j = 0; j < I.M; ++j) {
      br_from.push_back(D.bus0 + I.from[j]);
      br_to.push_back(D.bus0 + I.to[j]);
      br_kidx.push_back(-1);
      br_g.push_back(I.gsr[j]);
      br_b.push_back(I.bsr[j]);
      br_bc.push_back(I.bsr[j] + 0.5 * I.bch[j]);
      br_smax.push_back(I.smax[j]);
      br_sctg.push_back(I.sctg[j]);
      br_y.push_back(I.y[j]);
    }
    for (int k = 0; k < I.K; ++k) {
      br_kidx[D.br0 + I.ctg[k]] = k;
      ctg_br.push_back(D.br0 + I.ctg[k]);
    }
    for (int g = 0; g < I.G; ++g) {
      gen_bus.push_back(D.bus0 + I.gen_bus[g]);
      gen_zone.push_back(D.zone0 + I.gen_zone[g]);
      ga.push_back(I.ca[g]); gb.push_back(I.cb[g]); gcr.push_back(I.cr[g]); gpmax.push_back(I.pmax[g]);
      gramp.push_back(I.ramp[g]);
    }
    // CSR: bus -> branch ends, bus -> generators (entries in branch / generator order)
    std::vector<std::vector<int>> ends(I.n), gens(I.n), zg(I.Z);
    for (int j = 0; j < I.M; ++j) {
      ends[I.from[j]].push_back(((D.br0 + j) << 1) | 0);
      ends[I.to[j]].push_back(((D.br0 + j) << 1) | 1);
    }
    for (int g = 0; g < I.G; ++g) {
      gens[I.gen_bus[g]].push_back(D.gen0 + g);
      zg[I.gen_zone[g]].push_back(D.gen0 + g);
    }
    for (int i = 0; i < I.n; ++i) {
      inc.insert(inc.end(), ends[i].begin(), ends[i].end());
      inc_ptr.push_back((int)inc.size());
      bgen.insert(bgen.end(), gens[i].begin(), gens[i].end());
      bgen_ptr.push_back((int)bgen.size());
    }
    for (int z = 0; z < I.Z; ++z) {
      zgen.insert(zgen.end(), zg[z].begin(), zg[z].end());
      zgen_ptr.push_back((int)zgen.size());
    }
    load_p.insert(load_p.end(), I.load_p.begin(), I.load_p.end());
    load_q.insert(load_q.end(), I.load_q.begin(), I.load_q.end());
    rreq.insert(rreq.end(), I.rreq.begin(), I.rreq.end());
    dt.insert(dt.end(), I.dt.begin(), I.dt.end());
    zinv.insert(zinv.end(), I.zinv.begin(), I.zinv.end());
    z1.insert(z1.end(), I.z1.begin(), I.z1.end());
    lodf.insert(lodf.end(), I.lodf.begin(), I.lodf.end());
    // clip box: v, theta (ref pinned at 0), p, q, r
    const double inf = INFINITY;
    for (int t = 0; t < I.T; ++t)
      for (int i = 0; i < I.n; ++i) { lo.push_back(I.vmin[i]); hi.push_back(I.vmax[i]); }
    for (int t = 0; t < I.T; ++t)
      for (int i = 0; i < I.n; ++i) {
        lo.push_back(i == I.ref ? 0.0 : -inf);
        hi.push_back(i == I.ref ? 0.0 : inf);
      }
    for (int t = 0; t < I.T; ++t)
      for (int g = 0; g < I.G; ++g) { lo.push_back(I.pmin[g]); hi.push_back(I.pmax[g]); }
    for (int t = 0; t < I.T; ++t)
      for (int g = 0; g < I.G; ++g) { lo.push_back(I.qmin[g]); hi.push_back(I.qmax[g]); }
    for (int t = 0; t < I.T; ++t)
      for (int g = 0; g < I.G; ++g) { lo.push_back(0.0); hi.push_back(I.pmax[g]); }
  }
  int rc = 0;
  Inst *dinst;
  if ((rc = upload(h, &dinst, inst))) return rc;
  d.inst = dinst;
  d.n_inst = B;
  int *p;
  Real *r;
  Dc *z;
#define UPI(field, vec) if ((rc = upload(h, &p, vec))) return rc; d.field = p;
#define UPR(field, vec) { auto tmp_ = cast<Real>(vec); if ((rc = upload(h, &r, tmp_))) return rc; d.field = r; }
  UPI(br_from, br_from) UPI(br_to, br_to) UPI(br_kidx, br_kidx) UPI(gen_bus, gen_bus) UPI(gen_zone, gen_zone)
  UPI(inc_ptr, inc_ptr) UPI(inc, inc) UPI(bgen_ptr, bgen_ptr) UPI(bgen, bgen) UPI(zgen_ptr, zgen_ptr) UPI(zgen, zgen)
  UPI(ctg_br, ctg_br)
  UPR(br_g, br_g) UPR(br_b, br_b) UPR(br_bc, br_bc) UPR(br_smax, br_smax) UPR(br_sctg, br_sctg) UPR(br_y, br_y)
  UPR(gen_a, ga) UPR(gen_b, gb) UPR(gen_cr, gcr) UPR(gen_pmax, gpmax) UPR(gen_ramp, gramp)
  UPR(load_p, load_p) UPR(load_q, load_q) UPR(rreq, rreq) UPR(dt, dt) UPR(lo, lo) UPR(hi, hi)
#undef UPI
#undef UPR
  {
    auto zz = to_dc<Dc>(zinv);
    if ((rc = upload(h, &z, zz))) return rc;
    d.zinv = z;
    auto z1d = to_dc<Dc>(z1);
    if ((rc = upload(h, &z, z1d))) return rc;
    d.z1 = z;
  }
  // line-outage block in the requested storage type
  if (sizeof(Real) == 8) {
    double *q;
    if ((rc = upload(h, &q, lodf))) return rc;
    d.lodf = q;
  } else if (h->opt.lodf_dtype == QG_LODF_BF16) {
    std::vector<__nv_bfloat16> v(lodf.size());
    for (size_t i = 0; i < v.size(); ++i) v[i] = __float2bfloat16_rn((float)lodf[i]);
    __nv_bfloat16 *q;
    if ((rc = upload(h, &q, v))) return rc;
    d.lodf = q;
  } else if (h->opt.lodf_dtype == QG_LODF_BF16X2) {
    std::vector<__nv_bfloat162> v(lodf.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float f = (float)lodf[i];
      const __nv_bfloat16 hb = __float2bfloat16_rn(f);
      const __nv_bfloat16 lb = __float2bfloat16_rn(f - __bfloat162float(hb));
      v[i].x = hb;
      v[i].y = lb;
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
  d.c_p = (Real)h->opt.c_p; d.c_q = (Real)h->opt.c_q; d.c_s = (Real)h->opt.c_s; d.c_rz = (Real)h->opt.c_rz;
  d.rho = (Real)h->opt.rho; d.eps = (Real)h->opt.eps; d.beta = (Real)h->opt.beta;
  // work buffers
  long long sTM = 0, sTn = 0, sTZ = 0, sIB = 0, sPM = 0, sPK = 0;
  for (const Inst &I : inst) {
    sTM += (long long)I.T * I.M; sTn += (long long)I.T * I.n; sTZ += (long long)I.T * I.Z;
    sIB += (long long)I.T * I.n_ib; sPM += (long long)I.n_kt * I.T * I.M; sPK += (long long)I.n_mt * I.T * I.K;
  }
  Real *w;
  Dc *c;
#define WR(field, cnt) if ((rc = dalloc(h, &w, (size_t)(cnt)))) return rc; d.field = w;
#define WD(field, cnt) if ((rc = dalloc(h, &c, (size_t)(cnt)))) return rc; d.field = c;
  WR(pf, sTM) WR(qf, sTM) WR(pt, sTM) WR(qt, sTM) WR(qm2, sTM) WR(dP, sTn) WR(dQ, sTn) WR(dZ, sTZ)
  WR(pm, sPM) WR(pq, sPM) WR(pk, sPK) WR(avf, sTM) WR(avo, sTM) WR(ad, sTM)
  WD(pinj, sTn) WD(th, sTn) WD(w, sTn) WD(ginj, sTn) WD(mupart, sIB) WD(spart, sIB)
#undef WR
#undef WD
  unsigned char *qs;
  if ((rc = dalloc(h, &qs, (size_t)sTM))) return rc;
  d.qside = qs;
  double *op;
  if ((rc = dalloc(h, &op, (size_t)h->L.n_obj_slots * N_TERMS))) return rc;
  d.objp = op;
  d.obj = h->d_obj;
  d.terms = h->d_terms;
  d.g = static_cast<Real *>(h->d_g);
  d.step = h->d_step;
  return QG_OK;
}

int build_tables(qg_ctx *h) {
  std::vector<Blk> fwd1, fwd2, bus, bwd1, bwd2;
  std::vector<DcTile> dct;
  std::vector<CtgTile> ctt;
  for (int b = 0; b < h->n_inst; ++b) {
    const Inst &I = h->inst[b];
    for (int t = 0; t < I.T; ++t) {
      for (int j0 = 0; j0 < I.M; j0 += BLK) fwd1.push_back({R_BRANCH, b, t, j0, 0});
      for (int z0 = 0; z0 < I.Z; z0 += BLK) fwd1.push_back({R_ZONE, b, t, z0, 0});
      int ib = 0;
      for (int i0 = 0; i0 < I.n; i0 += BLK, ++ib) bus.push_back({R_BUS, b, t, i0, ib});
      for (int g0 = 0; g0 < I.G; g0 += BLK) bwd2.push_back({R_GEN, b, t, g0, 0});
    }
    for (int i0 = 0; i0 < I.n; i0 += 4) dct.push_back({b, i0});
    for (int mt = 0; mt < I.n_mt; ++mt)
      for (int kt = 0; kt < I.n_kt; ++kt) ctt.push_back({b, mt * 64, kt * 64, mt, kt});
  }
  fwd2 = bus;
  for (const Blk &x : fwd1)
    if (x.role == R_BRANCH) bwd1.push_back(x);
  std::vector<Blk> b2 = bus;
  b2.insert(b2.end(), bwd2.begin(), bwd2.end());
  bwd2 = b2;
  int rc;
  Blk *p;
  if ((rc = upload(h, &p, fwd1))) return rc; h->L.blk_fwd1 = p; h->L.n_fwd1 = (int)fwd1.size();
  if ((rc = upload(h, &p, fwd2))) return rc; h->L.blk_fwd2 = p; h->L.n_fwd2 = (int)fwd2.size();
  if ((rc = upload(h, &p, bus))) return rc; h->L.blk_adj1 = p; h->L.n_adj1 = (int)bus.size();
  if ((rc = upload(h, &p, bwd1))) return rc; h->L.blk_bwd1 = p; h->L.n_bwd1 = (int)bwd1.size();
  if ((rc = upload(h, &p, bwd2))) return rc; h->L.blk_bwd2 = p; h->L.n_bwd2 = (int)bwd2.size();
  DcTile *q;
  if ((rc = upload(h, &q, dct))) return rc; h->L.dct = q; h->L.n_dct = (int)dct.size();
  CtgTile *cq;
  if ((rc = upload(h, &cq, ctt))) return rc; h->L.ctt = cq; h->L.n_ctt = (int)ctt.size();
  // objective slots: one per block of fwd1, fwd2, ctg, bwd2
  std::vector<int> slot_inst;
  h->L.obj_fwd1 = (int)slot_inst.size();
  for (auto &x : fwd1) slot_inst.push_back(x.inst);
  h->L.obj_fwd2 = (int)slot_inst.size();
  for (auto &x : fwd2) slot_inst.push_back(x.inst);
  h->L.obj_ctg = (int)slot_inst.size();
  for (auto &x : ctt) slot_inst.push_back(x.inst);
  h->L.obj_bwd2 = (int)slot_inst.size();
  for (auto &x : bwd2) slot_inst.push_back(x.inst);
  h->L.n_obj_slots = (int)slot_inst.size();
  int *si;
  if ((rc = upload(h, &si, slot_inst))) return rc;
  h->L.slot_inst = si;
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

void free_all(qg_ctx *h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  for (auto &e : h->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
}

bool mixed(const qg_ctx *h) { return h->opt.precision == QG_MIXED; }

int run_eval(qg_ctx *h, const void *x) {
  cudaEvent_t *ev = h->profiling ? h->ev : nullptr;
  cudaError_t e = mixed(h) ? launch_eval<float, df32>(h->d32, h->L, x, h->maxT, ev)
                           : launch_eval<double, double>(h->d64, h->L, x, h->maxT, ev);
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("eval launch: ") + cudaGetErrorString(e));
  return QG_OK;
}

int run_adam(qg_ctx *h, void *x, void *m, void *v, double lr, double b1, double b2) {
  cudaError_t e;
  if (mixed(h))
    e = launch_adam<float>((float *)x, (float *)m, (float *)v, (const float *)h->d_g, h->d32.lo, h->d32.hi, h->n_x,
                           h->d_step, lr, b1, b2, h->opt.adam_eps, h->opt.adam_paper_eps, h->stream);
  else
    e = launch_adam<double>((double *)x, (double *)m, (double *)v, (const double *)h->d_g, h->d64.lo, h->d64.hi,
                            h->n_x, h->d_step, lr, b1, b2, h->opt.adam_eps, h->opt.adam_paper_eps, h->stream);
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
  g_create_error.clear();
  if (!out) return fail(nullptr, QG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_inst < 1 || !net || !hor || !ctg) return fail(nullptr, QG_ERR_INVALID_ARG, "bad batch arguments");
  qg_ctx *h = new qg_ctx();
  if (opt) h->opt = *opt;
  else qg_default_options(&h->opt);
  const qg_options &o = h->opt;
  if (o.precision != QG_FP64 && o.precision != QG_MIXED) { fail(h, QG_ERR_INVALID_ARG, "precision"); delete h; return QG_ERR_INVALID_ARG; }
  if (o.lodf_dtype < 0 || o.lodf_dtype > 2) { fail(h, QG_ERR_INVALID_ARG, "lodf_dtype"); delete h; return QG_ERR_INVALID_ARG; }
  if (!(o.eps >= 0) || !(o.beta >= 0) || !(o.c_p >= 0) || !(o.c_q >= 0) || !(o.c_s >= 0) || !(o.c_rz >= 0) ||
      !(o.rho >= 0) || !(o.adam_eps >= 0)) {
    fail(h, QG_ERR_INVALID_ARG, "penalty parameters must be finite and >= 0");
    delete h;
    return QG_ERR_INVALID_ARG;
  }
  int rc = QG_OK;
  h->n_inst = n_inst;
  h->hi.resize(n_inst);
  for (int b = 0; b < n_inst; ++b) {
    rc = read_instance(h, net[b], hor[b], ctg[b], h->hi[b], b);
    if (rc) { delete h; return rc; }
  }
  // dense inverse + line-outage block per instance, in parallel over instances
  {
    std::vector<int> rcs(n_inst, 0);
    std::vector<std::string> errs(n_inst);
    unsigned nth = std::max(1u, std::min((unsigned)n_inst, std::thread::hardware_concurrency()));
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
      if (rcs[b]) {
        fail(h, rcs[b], errs[b]);
        rc = rcs[b];
        delete h;
        return rc;
      }
  }
  // everything above is host-side validation and set-up; from here on the device is needed
  rc = check_device(h);
  if (rc) { delete h; return rc; }
  // instance descriptors
  long long x0 = 0, tb0 = 0, tm0 = 0, tg0 = 0, tz0 = 0, z0 = 0, l0 = 0, pm0 = 0, pk0 = 0, ib0 = 0;
  int bus0 = 0, br0 = 0, gen0 = 0, zone0 = 0, ctg0 = 0, tp0 = 0;
  for (int b = 0; b < n_inst; ++b) {
    const HostInst &I = h->hi[b];
    Inst D{};
    D.n = I.n; D.M = I.M; D.G = I.G; D.Z = I.Z; D.T = I.T; D.K = I.K; D.ref = I.ref;
    D.bus0 = bus0; D.br0 = br0; D.gen0 = gen0; D.zone0 = zone0; D.ctg0 = ctg0; D.tp0 = tp0;
    D.n_mt = (I.M + 63) / 64;
    D.n_kt = (I.K + 63) / 64;
    D.n_ib = (I.n + BLK - 1) / BLK;
    D.x0 = x0; D.tb0 = tb0; D.tm0 = tm0; D.tg0 = tg0; D.tz0 = tz0; D.z0 = z0; D.l0 = l0;
    D.pm0 = pm0; D.pk0 = pk0; D.ib0 = ib0;
    D.wfloor_ctg = o.c_s * o.beta * o.eps * ((double)I.M * I.K - I.K);
    D.inv_n = 1.0 / I.n;
    df32 s = split(D.inv_n);
    D.inv_n_hi = s.hi; D.inv_n_lo = s.lo;
    h->inst.push_back(D);
    x0 += (long long)I.T * (2LL * I.n + 3LL * I.G);
    tb0 += (long long)I.T * I.n; tm0 += (long long)I.T * I.M; tg0 += (long long)I.T * I.G; tz0 += (long long)I.T * I.Z;
    z0 += (long long)I.n * I.n; l0 += (long long)I.M * I.K;
    pm0 += (long long)D.n_kt * I.T * I.M; pk0 += (long long)D.n_mt * I.T * I.K; ib0 += (long long)I.T * D.n_ib;
    bus0 += I.n; br0 += I.M; gen0 += I.G; zone0 += I.Z; ctg0 += I.K; tp0 += I.T;
    h->maxT = std::max(h->maxT, I.T);
  }
  h->n_x = x0;
  h->L.n_x = x0;
  h->L.lodf_dtype = o.precision == QG_MIXED ? o.lodf_dtype : QG_LODF_F32;
  h->L.stream = nullptr;
  const size_t rs = mixed(h) ? sizeof(float) : sizeof(double);
  if ((rc = build_tables(h)) || (rc = dalloc(h, &h->d_obj, (size_t)n_inst)) ||
      (rc = dalloc(h, &h->d_terms, (size_t)n_inst * N_TERMS)) || (rc = dalloc(h, (char **)&h->d_g, rs * h->n_x)) ||
      (rc = dalloc(h, (char **)&h->d_m, rs * h->n_x)) || (rc = dalloc(h, (char **)&h->d_v, rs * h->n_x)) ||
      (rc = dalloc(h, (char **)&h->d_xs, rs * h->n_x)) || (rc = dalloc(h, &h->d_xd, (size_t)h->n_x)) ||
      (rc = dalloc(h, &h->d_step, 1))) {
    free_all(h);
    delete h;
    return rc;
  }
  if (cudaMemset(h->d_step, 0, sizeof(long long)) != cudaSuccess ||
      cudaMemset(h->d_m, 0, rs * h->n_x) != cudaSuccess || cudaMemset(h->d_v, 0, rs * h->n_x) != cudaSuccess) {
    fail(h, QG_ERR_CUDA, "cudaMemset");
    free_all(h);
    delete h;
    return QG_ERR_CUDA;
  }
  rc = mixed(h) ? build_device<float, df32>(h, h->d32) : build_device<double, double>(h, h->d64);
  if (!rc) {
    cudaError_t e = mixed(h) ? prepare_eval<float, df32>(h->maxT) : prepare_eval<double, double>(h->maxT);
    if (e != cudaSuccess) rc = fail(h, QG_ERR_CUDA, std::string("prepare_eval: ") + cudaGetErrorString(e));
  }
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  // host copies no longer needed beyond sizes
  for (auto &I : h->hi) {
    I.zinv.clear(); I.zinv.shrink_to_fit();
    I.lodf.clear(); I.lodf.shrink_to_fit();
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

int qg_layout(const qg_ctx *h, int32_t inst, int64_t *first, int64_t *n_x, int64_t offsets[5]) {
  if (!h || inst < 0 || inst >= h->n_inst) return QG_ERR_INVALID_ARG;
  const Inst &I = h->inst[inst];
  const int64_t Tn = (int64_t)I.T * I.n, TG = (int64_t)I.T * I.G;
  if (first) *first = I.x0;
  if (n_x) *n_x = 2 * Tn + 3 * TG;
  if (offsets) {
    offsets[0] = 0; offsets[1] = Tn; offsets[2] = 2 * Tn; offsets[3] = 2 * Tn + TG; offsets[4] = 2 * Tn + 2 * TG;
  }
  return QG_OK;
}

int qg_set_stream(qg_ctx *h, void *stream) {
  if (!h) return QG_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  h->L.stream = h->stream;
  return QG_OK;
}

int qg_eval_grad(qg_ctx *h, const void *x, double *obj, void *g) {
  if (!h || !x) return h ? fail(h, QG_ERR_INVALID_ARG, "x is NULL") : QG_ERR_INVALID_ARG;
  int rc = run_eval(h, x);
  if (rc) return rc;
  const size_t rs = mixed(h) ? sizeof(float) : sizeof(double);
  if (obj) CUDA_TRY(h, cudaMemcpyAsync(obj, h->d_obj, sizeof(double) * h->n_inst, cudaMemcpyDeviceToDevice, h->stream));
  if (g) CUDA_TRY(h, cudaMemcpyAsync(g, h->d_g, rs * h->n_x, cudaMemcpyDeviceToDevice, h->stream));
  return QG_OK;
}

int qg_eval_grad_host(qg_ctx *h, const double *x, double *obj, double *g) {
  if (!h || !x) return h ? fail(h, QG_ERR_INVALID_ARG, "x is NULL") : QG_ERR_INVALID_ARG;
  const long long n = h->n_x;
  const int nb = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  if (mixed(h)) {
    CUDA_TRY(h, cudaMemcpyAsync(h->d_xd, x, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    k_d2f<<<nb, 256, 0, h->stream>>>(h->d_xd, (float *)h->d_xs, n);
  } else {
    CUDA_TRY(h, cudaMemcpyAsync(h->d_xs, x, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  }
  int rc = run_eval(h, h->d_xs);
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
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaGetLastError());
  return QG_OK;
}

int qg_adam_step(qg_ctx *h, void *x, void *m, void *v, double lr, double beta1, double beta2) {
  if (!h || !x || !m || !v) return h ? fail(h, QG_ERR_INVALID_ARG, "null pointer") : QG_ERR_INVALID_ARG;
  if (!(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1))
    return fail(h, QG_ERR_INVALID_ARG, "Adam parameters out of range");
  return run_adam(h, x, m, v, lr, beta1, beta2);
}

int qg_solve(qg_ctx *h, void *x, int32_t iters, double lr, double beta1, double beta2, double *obj_trace) {
  if (!h || !x || iters < 0) return h ? fail(h, QG_ERR_INVALID_ARG, "bad solve arguments") : QG_ERR_INVALID_ARG;
  if (!(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1))
    return fail(h, QG_ERR_INVALID_ARG, "Adam parameters out of range");
  if (iters == 0) return QG_OK;
  const bool same = h->gexec && h->g_x == x && h->g_lr == lr && h->g_b1 == beta1 && h->g_b2 == beta2;
  if (!same) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    cudaStream_t cs;
    CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = h->stream;
    h->stream = cs;
    h->L.stream = cs;
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = QG_OK;
    if (e == cudaSuccess) {
      rc = run_eval(h, x);
      if (!rc) rc = run_adam(h, x, h->d_m, h->d_v, lr, beta1, beta2);
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (!rc && e2 == cudaSuccess) {
        e = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
      } else if (!rc) {
        e = e2;
      }
    }
    h->stream = saved;
    h->L.stream = saved;
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    h->g_x = x; h->g_lr = lr; h->g_b1 = beta1; h->g_b2 = beta2;
  }
  for (int it = 0; it < iters; ++it) {
    CUDA_TRY(h, cudaGraphLaunch(h->gexec, h->stream));
    if (obj_trace)
      CUDA_TRY(h, cudaMemcpyAsync(obj_trace + (size_t)it * h->n_inst, h->d_obj, sizeof(double) * h->n_inst,
                                  cudaMemcpyDeviceToDevice, h->stream));
  }
  return QG_OK;
}

int qg_breakdown(qg_ctx *h, double *out) {
  if (!h || !out) return QG_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(out, h->d_terms, sizeof(double) * N_TERMS * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
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

int qg_set_profiling(qg_ctx *h, int on) {
  if (!h) return QG_ERR_INVALID_ARG;
  if (on && !h->ev[0])
    for (auto &e : h->ev) CUDA_TRY(h, cudaEventCreate(&e));
  if ((bool)on != h->profiling && h->gexec) {  // the cached graph must be re-captured
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  h->profiling = on != 0;
  return QG_OK;
}

int qg_phase_times(qg_ctx *h, float *ms, int32_t cap) {
  if (!h || !ms || cap < 0) return QG_ERR_INVALID_ARG;
  if (!h->profiling) return fail(h, QG_ERR_INVALID_ARG, "profiling is off");
  CUDA_TRY(h, cudaEventSynchronize(h->ev[N_PHASES - 1]));
  int n = 0;
  for (int k = 0; k < N_PHASES && k < cap; ++k) {
    float v = 0.f;
    cudaEvent_t end = h->ev[k + 1];
    if (k == N_PHASES - 1 && cudaEventQuery(end) != cudaSuccess) break;
    if (cudaEventElapsedTime(&v, h->ev[k], end) != cudaSuccess) v = -1.f;
    ms[n++] = v;
  }
  cudaGetLastError();
  return n;
}

const char *qg_last_error(const qg_ctx *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int qg_version(void) { return 100; }

}  // extern "C"
