// Device kernels of one QuasiGrad objective + gradient evaluation (Sec. II,
// Eq. grads) and of the projected Adam step (Alg. 3), for GB300 (sm_103a).
//
// One evaluation is five fused stage kernels; every block reads its role,
// instance and period from spans passed as kernel parameters, so one launch
// mixes independent work and serves uneven batched instances:
//   s1  branch flows (pi model) + thermal penalty | zonal reserve sums |
//       base DC flows f = PTDF_G p_G - PTDF load - mean(p_inj) PTDF 1
//       (sparse DC mode: flows from the angles of the forward solve)
//   s2  bus P/Q balance by warp-segmented CSR reduction + soft-abs penalty |
//       contingency flows F = f_m + L[m,k] f_k, overload penalty and both
//       backward sums (the SMW rank-1 correction of Eq. rank_correct in flow space)
//   s3  dz/df summed over contingency tiles; branch-end adjoints (chain rule) |
//       folds of the stage-1/2 objective slots
//   s4  bus gather of branch-end adjoints (warp-segmented) -> g_v, g_theta
//       [+ fused Adam] | adjoint DC products PTDF_G^T dz/df (Eq. 2nd_lin_sys)
//       (sparse DC mode: the right-hand side of the adjoint solve)
//   s5  device terms (costs and values, limits, ramps, on-status) and gradients
//       incl. the slack-corrected injection adjoint eta - mean(eta) (Eq.
//       correction) [+ fused Adam] | transformer gradients; the last block
//       reduces the objective and advances the Adam step counter.
// Sparse DC mode: k_sp_inj, k_sp_fwd, k_sp_tail, k_sp_back solve Yhat theta = b
// through the sparse factor with a dense tail, before s1 and after s4.
// No floating-point atomics: every sum has a fixed order, so repeated
// evaluations are bitwise identical.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdint>
#include <utility>
#include <vector>

#include "qg_internal.h"

namespace qg {

// ---------------------------------------------------------------------------------------------
// index-checked build (QG_CHECK_BOUNDS): the build step rewrites every d.<array>[i] of this file
// as qg_at(d.<array>, i, __LINE__), which checks the element's address against the registered
// device arrays
// ---------------------------------------------------------------------------------------------

#ifdef QG_CHECK_BOUNDS
constexpr int QG_MAX_RANGES = 8192;
struct QgRange {
  unsigned long long lo, hi;  // [lo, hi)
};
__device__ QgRange g_qg_ranges[QG_MAX_RANGES];  // sorted by lo, disjoint
__device__ int g_qg_nranges;
__device__ int g_qg_bad_line;                 // first failing access: its source line (0: none)
__device__ unsigned long long g_qg_bad_addr;  // and its address
__device__ __align__(16) unsigned char g_qg_dummy[64];

template <typename T>
__device__ __forceinline__ T &qg_at(T *p, long long i, int line) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p + i);
  int lo = 0, hi = g_qg_nranges - 1;
  while (lo <= hi) {  // the last range starting at or below a
    const int mid = (lo + hi) >> 1;
    if (g_qg_ranges[mid].lo <= a) lo = mid + 1;
    else hi = mid - 1;
  }
  if (hi >= 0 && a + sizeof(T) <= g_qg_ranges[hi].hi) return p[i];
  if (atomicCAS(&g_qg_bad_line, 0, line) == 0) g_qg_bad_addr = a;
  return *reinterpret_cast<T *>(g_qg_dummy);
}

namespace {
std::mutex g_ranges_mu;
std::map<unsigned long long, unsigned long long> g_ranges;  // base -> bytes, every live registration

void upload_ranges() {
  std::vector<QgRange> v;
  for (const auto &r : g_ranges) v.push_back({r.first, r.first + r.second});
  if (v.size() > (size_t)QG_MAX_RANGES) v.resize(QG_MAX_RANGES);
  const int n = (int)v.size();
  cudaDeviceSynchronize();  // no kernel reads the table while it changes (debug build)
  if (n) cudaMemcpyToSymbol(g_qg_ranges, v.data(), sizeof(QgRange) * n);
  cudaMemcpyToSymbol(g_qg_nranges, &n, sizeof(int));
}
}  // namespace

void bounds_register(const void *p, size_t bytes) {
  if (!p || !bytes) return;
  std::lock_guard<std::mutex> lock(g_ranges_mu);
  auto &b = g_ranges[reinterpret_cast<unsigned long long>(p)];
  if (b == bytes) return;
  b = bytes;
  upload_ranges();
}

void bounds_unregister(const void *p) {
  std::lock_guard<std::mutex> lock(g_ranges_mu);
  if (g_ranges.erase(reinterpret_cast<unsigned long long>(p))) upload_ranges();
}

int bounds_report(long long *line, unsigned long long *addr) {
  int l = 0;
  unsigned long long a = 0;
  cudaDeviceSynchronize();
  cudaMemcpyFromSymbol(&l, g_qg_bad_line, sizeof(int));
  cudaMemcpyFromSymbol(&a, g_qg_bad_addr, sizeof(a));
  if (line) *line = l;
  if (addr) *addr = a;
  return l ? 1 : 0;
}
#else
void bounds_register(const void *, size_t) {}
void bounds_unregister(const void *) {}
int bounds_report(long long *line, unsigned long long *addr) {
  if (line) *line = 0;
  if (addr) *addr = 0;
  return -1;
}
#endif

// ---------------------------------------------------------------------------------------------
// double-FP32 arithmetic (Knuth's TwoSum, FMA-based TwoProd)
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, e);
  return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}

// acc += a * b (a, b double-FP32; the lo * lo term is below the format's precision)
__device__ __forceinline__ void df_mac(df32 &acc, df32 a, df32 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, e;
  two_sum(acc.hi, p, s, e);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

template <typename Dc>
struct DcOps;

template <>
struct DcOps<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double from_real(double v) { return v; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double neg(double a) { return -a; }
  __device__ static void mac(double &acc, double a, double b) { acc = fma(a, b, acc); }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double inv_n(const Inst &I) { return I.inv_n; }
  __device__ static double to_real(double a) { return a; }
  __device__ static float to_float(double a) { return (float)a; }
  __device__ static double shfl_down(double a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
  __device__ static double bcast(double a) { return __shfl_sync(0xffffffffu, a, 0); }
};

template <>
struct DcOps<df32> {
  __device__ static df32 zero() { return {0.f, 0.f}; }
  __device__ static df32 from_real(float v) { return {v, 0.f}; }
  __device__ static df32 add(df32 a, df32 b) { return df_add(a, b); }
  __device__ static df32 neg(df32 a) { return {-a.hi, -a.lo}; }
  __device__ static void mac(df32 &acc, df32 a, df32 b) { df_mac(acc, a, b); }
  __device__ static df32 mul(df32 a, df32 b) {
    df32 r = {0.f, 0.f};
    df_mac(r, a, b);
    return r;
  }
  __device__ static df32 inv_n(const Inst &I) {
    const float h = (float)I.inv_n;
    return {h, (float)(I.inv_n - (double)h)};
  }
  __device__ static float to_real(df32 a) { return __fadd_rn(a.hi, a.lo); }
  __device__ static float to_float(df32 a) { return __fadd_rn(a.hi, a.lo); }
  __device__ static df32 shfl_down(df32 a, int o) {
    return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
  }
  __device__ static df32 bcast(df32 a) { return {__shfl_sync(0xffffffffu, a.hi, 0), __shfl_sync(0xffffffffu, a.lo, 0)}; }
};

__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(df32 a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ double dsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float dsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ void dsincos(double a, double *s, double *c) { sincos(a, s, c); }
__device__ __forceinline__ void dsincos(float a, float *s, float *c) { sincosf(a, s, c); }

__device__ __forceinline__ double drsqrt(double v) { return rsqrt(v); }
__device__ __forceinline__ float drsqrt(float v) { return rsqrtf(v); }

// sqrt(a) and w / sqrt(a) for a >= 0.  Finite a > 0: through one reciprocal square root r (CUDA's
// rsqrt: a few ulp), the value a r and the factor w r, where the square root and the division would
// each be a long FP64 sequence on GB300's FP64 pipe; a = 0 gives (0, 0); +inf and NaN take the plain
// square root and division, so that they propagate as they would there.
template <typename Real>
__device__ __forceinline__ void root_and_ratio(Real a, Real w, Real &s, Real &q) {
  if (a == Real(0)) {
    s = Real(0);
    q = Real(0);
  } else if (a < Real(INFINITY)) {
    const Real r = drsqrt(a);
    s = a * r;
    q = w * r;
  } else {
    s = dsqrt(a);
    q = w / s;
  }
}

// soft-ReLU sigma_s(u) = sqrt(max(u,0)^2 + eps^2) and its derivative max(u,0) / sigma_s(u)
// (Sec. II-C footnote)
template <typename Real>
__device__ __forceinline__ void soft_relu(Real u, Real eps, Real &val, Real &der) {
  const Real m = u > Real(0) ? u : Real(0);
  root_and_ratio(m * m + eps * eps, m, val, der);
}

// soft-abs |u|_s = sqrt(u^2 + eps^2) and its derivative u / |u|_s
template <typename Real>
__device__ __forceinline__ void soft_abs(Real u, Real eps, Real &val, Real &der) {
  root_and_ratio(u * u + eps * eps, u, val, der);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of NV doubles; result valid in thread 0.
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
  __shared__ double red[NTHR / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[wid][k] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < NTHR / 32 ? red[lane][k] : 0.0);
  }
  __syncthreads();
}

// Deterministic block sum of one Dc value; result valid in thread 0.
template <typename Dc>
__device__ Dc block_sum_dc(Dc v) {
  __shared__ Dc red[NTHR / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = DcOps<Dc>::add(v, DcOps<Dc>::shfl_down(v, o));
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    Dc s = lane < NTHR / 32 ? red[lane] : DcOps<Dc>::zero();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = DcOps<Dc>::add(s, DcOps<Dc>::shfl_down(s, o));
    v = s;
  }
  __syncthreads();
  return v;
}

// Objective terms of one block: at most three per role, accumulated in the DC product type
// (double, or double-FP32 on the mixed path: no FP64 arithmetic there).
template <typename Dc>
struct Obj3 {
  Dc v[3];
  int id[3];  // term ids, -1 when unused
};

template <typename Dc>
__device__ __forceinline__ Obj3<Dc> obj3(int a, int b = -1, int c = -1) {
  Obj3<Dc> o;
  o.v[0] = o.v[1] = o.v[2] = DcOps<Dc>::zero();
  o.id[0] = a;
  o.id[1] = b;
  o.id[2] = c;
  return o;
}

// Deterministic block sum of the three terms; thread 0 writes the block's slot (zeros elsewhere).
template <typename Dc>
__device__ void write_obj(Dc *objp, int slot, Obj3<Dc> o) {
  __shared__ Dc red[NTHR / 32][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) o.v[k] = DcOps<Dc>::add(o.v[k], DcOps<Dc>::shfl_down(o.v[k], q));
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) red[wid][k] = o.v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Dc v = lane < NTHR / 32 ? red[lane][k] : DcOps<Dc>::zero();
#pragma unroll
      for (int q = 16; q > 0; q >>= 1) v = DcOps<Dc>::add(v, DcOps<Dc>::shfl_down(v, q));
      o.v[k] = v;
    }
    if (lane == 0) {
      Dc *dst = objp + (long long)slot * N_TERMS;
#pragma unroll
      for (int k = 0; k < N_TERMS; ++k) dst[k] = DcOps<Dc>::zero();
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (o.id[k] >= 0) dst[o.id[k]] = o.v[k];
    }
  }
}

// Programmatic dependent launch: a stage may begin as its predecessor's blocks exit and waits
// (griddepcontrol.wait) for the predecessor's completion before reading its results; loads of
// data no earlier stage writes come before the wait.  No stage triggers its dependents early:
// blocks of the next stage parked at the wait slowed the long sparse-solve kernels (measured).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ float f_nan() { return __int_as_float(0x7fc00000); }

// Two FP32 values in one 64-bit register pair (x in the low half) and the sm_100+ paired FMA on
// them: each half is rounded exactly as a scalar fma.rn of the same operands would be.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// max of three FP32 values (sm_100+); like fmaxf, a NaN operand is ignored
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// min of three FP32 values (sm_100+); like fminf, a NaN operand is ignored
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

struct Where {
  int role, inst, t, sub;
};

// Penalty smoothing eps and homotopy scale beta of this evaluation (Sec. II-F): the handle's options,
// or iteration i of a scheduled solve (i counted from the step at the start of that solve).
template <typename Real>
struct HP {
  Real eps, beta;
};

template <typename Real, typename Dc>
__device__ __forceinline__ long long sched_index(const Dev<Real, Dc> &d) {
  long long it = *d.step + d.step_off - *d.trace_step0;
  return it < 0 ? 0 : (it >= d.sched_len ? d.sched_len - 1 : it);
}

template <typename Real, typename Dc>
__device__ __forceinline__ HP<Real> hparams(const Dev<Real, Dc> &d) {
  if (!d.sched) return {d.eps, d.beta};
  const long long it = sched_index(d);
  return {(Real)d.sched[3 * it + 1], (Real)d.sched[3 * it + 2]};
}

// Block -> (role, instance, period or period chunk, slice) by binary search over the spans.
__device__ __forceinline__ Where locate(const Spans &S) {
  const int bid = blockIdx.x;
  int lo = 0, hi = S.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S.s[mid].first <= bid) lo = mid;
    else hi = mid - 1;
  }
  const Span &sp = S.s[lo];
  const int rel = bid - sp.first;
  return {sp.role, sp.inst, rel / sp.per_t, rel % sp.per_t};
}

// Warp-segmented inclusive sum over a warp pack whose rows are contiguous runs of lanes.
// Returns true in the last lane of each row (where the row total sits).
template <typename Real>
__device__ __forceinline__ bool seg_sum2(int row, Real &a, Real &b) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const Real a2 = __shfl_up_sync(0xffffffffu, a, d);
    const Real b2 = __shfl_up_sync(0xffffffffu, b, d);
    const int r2 = __shfl_up_sync(0xffffffffu, row, d);
    if (lane >= d && r2 == row) {
      a += a2;
      b += b2;
    }
  }
  const int rn = __shfl_down_sync(0xffffffffu, row, 1);
  return lane == 31 || rn != row;
}

// Tap ratio and phase shift of branch j (local id) in period t: the transformer variables, or
// (1, 0) on lines.
template <typename Real, typename Dc>
__device__ __forceinline__ void branch_tap(const Dev<Real, Dc> &d, const Inst &I, int t, int jg,
                                           const Real *__restrict__ x, Real &tau, Real &phi, int &xi) {
  xi = d.br_xf[jg];
  tau = Real(1);
  phi = Real(0);
  if (xi >= 0) {
    const long long k = I.xtau0 + (long long)t * I.X + xi;
    tau = x[k];
    phi = x[k + (long long)I.T * I.X];
  }
}

// ---------------------------------------------------------------------------------------------
// stage 1
// ---------------------------------------------------------------------------------------------

constexpr int GBC = 128;  // generator-bus chunk of the DC products

// Pi-model flows at both ends of branch jg (global id) in period t (Sec. II-F line-flow example): a
// transformer's tap enters through v_f / tau, its phase shift through d = theta_f - theta_o - phi.
// Written without the cancellation of g vf^2 against g vf vo cos(d) (vf standing for v_f / tau):
//   p_fr = g vf (vf - vo) + g vf vo (1 - cos d) - b vf vo sin d,  and likewise for the others,
// with 1 - cos d = sin^2 d / (1 + cos d) while cos d > 0.
template <typename Real, typename Dc>
__device__ __forceinline__ void pi_flow(const Dev<Real, Dc> &d, const Inst &I, int t, int jg, const Real *__restrict__ x,
                                        Real &pf, Real &qf, Real &pt, Real &qt) {
  const int2 ft = d.br_end[jg];
  const Real *v = x + I.x0 + (long long)t * I.n;
  const Real *th = v + (long long)I.T * I.n;
  Real tau, phi;
  int xi;
  branch_tap(d, I, t, jg, x, tau, phi, xi);
  const Real vf = v[ft.x] / tau, vo = v[ft.y];
  const Real dl = th[ft.x] - th[ft.y] - phi;
  const Real g = d.br_g[jg], bb = d.br_b[jg], hch = d.br_hch[jg];
  Real sn, cs;
  dsincos(dl, &sn, &cs);
  const Real vv = vf * vo;
  const Real dv = vf - vo;
  const Real omc = cs > Real(0) ? sn * sn / (Real(1) + cs) : Real(1) - cs;
  pf = g * vf * dv + g * vv * omc - bb * vv * sn;
  pt = -g * vo * dv + g * vv * omc + bb * vv * sn;
  qf = -bb * vf * dv - hch * vf * vf - bb * vv * omc - g * vv * sn;
  qt = bb * vo * dv - hch * vo * vo - bb * vv * omc + g * vv * sn;
}

template <typename Real, typename Dc>
__device__ void s1_branch(const Dev<Real, Dc> &d, const Inst &I, int t, int sub, const Real *__restrict__ x,
                          Obj3<Dc> &acc, const HP<Real> hp) {
  const int j = sub * NTHR + threadIdx.x;
  if (j >= I.M) return;
  const int jg = I.br0 + j;
  const Real smax = d.br_smax[jg];
  const Real wt = d.dt[I.tp0 + t] * d.c_s * hp.beta;  // loaded before the stores below
  Real pf, qf, pt, qt;
  pi_flow(d, I, t, jg, x, pf, qf, pt, qt);
  const long long e = I.tm0 + (long long)t * I.M + j;
  d.pf[e] = pf;
  d.qf[e] = qf;
  d.pt[e] = pt;
  d.qt[e] = qt;
  const Real qf2 = qf * qf, qt2 = qt * qt;
  const bool qto = qt2 > qf2;  // ties go to the "fr" end
  d.qm2[e] = qto ? qt2 : qf2;
  d.qside[e] = qto ? 1 : 0;
  // thermal penalty on the worse end (Example 1)
  const Real sm2 = fmax(pf * pf + qf * qf, pt * pt + qt * qt);
  Real val = hp.eps;
  if (sm2 > smax * smax) {
    Real der;
    soft_relu(dsqrt(sm2) - smax, hp.eps, val, der);
  }
  acc.v[0] = DcOps<Dc>::from_real(wt * val);
}

// Zonal reserve shortfall of zone `sub` in period t: the block sums the zone's reserve
// offers (fixed order, FP64 in both paths), then sigma_s(R_zt - sum r) and its derivative.
template <typename Real, typename Dc>
__device__ void s1_zone(const Dev<Real, Dc> &d, const Inst &I, int t, int z, const Real *__restrict__ x,
                        Obj3<Dc> &acc, const HP<Real> hp) {
  __shared__ double red[NTHR / 32];
  const int zg = I.zone0 + z;  // global zone id; zgen_ptr is one CSR over all zones of the batch
  const Real *r = x + I.x0 + 2LL * I.T * I.n + 2LL * I.T * I.G + (long long)t * I.G;
  const long long k = I.tz0 + (long long)t * I.Z + z;
  double req = 0;
  Real w = 0;
  if (threadIdx.x == 0) {  // loaded ahead of the sum (no dependence on it)
    req = d.lim_rreq[k];
    w = d.dt[I.tp0 + t] * d.c_rz * hp.beta;
  }
  const int e0 = d.zgen_ptr[zg], e1 = d.zgen_ptr[zg + 1];
  double sr = 0;
  for (int e = e0 + threadIdx.x; e < e1; e += NTHR) sr += (double)r[d.zgen[e] - I.gen0];
  sr = warp_sum(sr);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0;
#pragma unroll
    for (int q = 0; q < NTHR / 32; ++q) tot += red[q];
    Real val, der;
    soft_relu(Real(req - tot), hp.eps, val, der);
    d.dZ[k] = w * der;
    acc.v[0] = DcOps<Dc>::from_real(w * val);
  }
}

// Dispatch (and on-status) snapshot for the ramp (and startup / shutdown) terms of a fused Adam
// update (stage 5 reads the pre-update p, u of the neighbouring periods): the periods [t0, t0 + 8)
// of a DC-flow block row, split evenly over the row's blocks.
template <typename Real, typename Dc>
__device__ __forceinline__ void pold_share(const Dev<Real, Dc> &d, const Inst &I, int t0, int sub,
                                           const Real *__restrict__ x) {
  const int tn = min(DCF_TC, I.T - t0);
  const int n = tn * I.G, nsub = (I.M + DCF_BM - 1) / DCF_BM;
  const int per = (n + nsub - 1) / nsub;
  const int lo = min(n, sub * per), hi = min(n, lo + per);
  const long long base = (long long)t0 * I.G;
  const Real *p = x + I.x0 + 2LL * I.T * I.n;
  for (int e = lo + threadIdx.x; e < hi; e += NTHR) d.pold[I.tg0 + base + e] = p[base + e];
  if (I.uc)
    for (int e = lo + threadIdx.x; e < hi; e += NTHR) d.uold[I.tg0 + base + e] = x[I.xu0 + base + e];
}

// Base DC flows of branches [m0, m0+32) in periods [t0, t0+8):
//   f[t,m] = sum_gb PTDF_G[m,gb] p_G[t,gb] - (PTDF load_t)[m] - mu_t (PTDF 1)[m],
//   mu_t = (sum_g p[t,g] - load_t) / n   (uniform slack, Sec. II-E).
template <typename Real, typename Dc>
__device__ void s1_dcf(const Dev<Real, Dc> &d, const Inst &I, int tc, int sub, const Real *__restrict__ x) {
  __shared__ Dc s_pg[DCF_TC][GBC + 1];
  __shared__ Dc s_pt[DCF_BM][GBC + 1];
  __shared__ Dc s_mu[DCF_TC];
  const int t0 = tc * DCF_TC, m0 = sub * DCF_BM;
  const int tl = threadIdx.x >> 5, ml = threadIdx.x & 31;
  const int t = t0 + tl, m = m0 + ml;
  const Real *p = x + I.x0 + 2LL * I.T * I.n;
  // the output's own terms first (none depends on the products): load latency overlaps the products
  const bool out = t < I.T && m < I.M;
  const long long e = I.tm0 + (long long)(out ? t : 0) * I.M + (out ? m : 0);
  const Dc cl = d.cload[e], rs = d.rsum[I.br0 + (out ? m : 0)];
  const Dc lt = d.ltot[I.tp0 + (t < I.T ? t : 0)];
  const int xi = d.br_xf[I.br0 + (out ? m : 0)], kx = d.br_kidx[I.br0 + (out ? m : 0)];
  const Real bphi = (out && xi >= 0) ? d.br_b[I.br0 + m] * x[I.xtau0 + (long long)(I.T + t) * I.X + xi] : Real(0);
  Dc acc = DcOps<Dc>::zero();
  Dc tot = DcOps<Dc>::zero();  // running sum of p_G over generator buses for mu_t (warp tl)
  // columns: generator buses (their dispatch), then transformers (their phase-shift flow b = b_sr phi)
  for (int c0 = 0; c0 < I.Gc; c0 += GBC) {
    const int cn = min(GBC, I.Gc - c0);
    if (c0 > 0) __syncthreads();  // the previous chunk's products are done with s_pt, s_pg
    // the PTDF tile first, as asynchronous copies to shared memory: they proceed during the gather
#pragma unroll 8
    for (int e = threadIdx.x; e < DCF_BM * cn; e += NTHR) {
      const int r = e / cn, c = e % cn;
      if (m0 + r < I.M) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&s_pt[r][c]);
        const Dc *src = d.ptdfg + I.pg0 + (long long)(m0 + r) * I.Gc + c0 + c;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
      } else {
        s_pt[r][c] = DcOps<Dc>::zero();
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // the signed dispatch of each generator bus in the block's periods: round 1 loads each entry's
    // first device and device count (static), round 2 its dispatch; a thread's entries are all in
    // flight together; further devices of a bus (rare) take more rounds
    constexpr int EPT = (DCF_TC * GBC + NTHR - 1) / NTHR;
    int dv[EPT], dn[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + k * NTHR, r = e / cn, c = e - r * cn;
      const bool gen = e < DCF_TC * cn && t0 + r < I.T && c0 + c < I.Gb;
      dv[k] = gen ? d.gb_dev0[I.gb0 + c0 + c] : -1;
      dn[k] = gen ? d.gb_ndev[I.gb0 + c0 + c] : 0;
    }
    Real pv[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + k * NTHR, r = e / cn;
      pv[k] = dv[k] >= 0 ? d.gen_sgn[dv[k]] * p[(long long)(t0 + r) * I.G + (dv[k] - I.gen0)] : Real(0);
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + k * NTHR, r = e / cn, c = e - r * cn, tt = t0 + r, cc = c0 + c;
      if (e >= DCF_TC * cn) break;
      Dc s = DcOps<Dc>::zero();
      if (dv[k] >= 0) {  // producers add, consumers subtract (CSR order)
        s = DcOps<Dc>::from_real(pv[k]);
        if (dn[k] > 1) {
          const int q0 = d.gb_ptr[I.gb0 + cc];
          for (int q = q0 + 1; q < q0 + dn[k]; ++q) {
            const int gq = d.gb_gen[q];
            s = DcOps<Dc>::add(s, DcOps<Dc>::from_real(d.gen_sgn[gq] * p[(long long)tt * I.G + (gq - I.gen0)]));
          }
        }
      } else if (tt < I.T && cc >= I.Gb) {  // a transformer column
        const int xi = cc - I.Gb;
        const Real phi = x[I.xtau0 + (long long)(I.T + tt) * I.X + xi];
        s = DcOps<Dc>::from_real(d.br_b[I.br0 + d.xf_br[I.xf0 + xi]] * phi);
      }
      s_pg[r][c] = s;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    {  // four independent accumulation chains (the double-FP32 add is a long dependency)
      Dc a1 = DcOps<Dc>::zero(), a2 = DcOps<Dc>::zero(), a3 = DcOps<Dc>::zero();
      int c = 0;
      for (; c + 4 <= cn; c += 4) {
        DcOps<Dc>::mac(acc, s_pt[ml][c], s_pg[tl][c]);
        DcOps<Dc>::mac(a1, s_pt[ml][c + 1], s_pg[tl][c + 1]);
        DcOps<Dc>::mac(a2, s_pt[ml][c + 2], s_pg[tl][c + 2]);
        DcOps<Dc>::mac(a3, s_pt[ml][c + 3], s_pg[tl][c + 3]);
      }
      for (; c < cn; ++c) DcOps<Dc>::mac(acc, s_pt[ml][c], s_pg[tl][c]);
      acc = DcOps<Dc>::add(acc, DcOps<Dc>::add(DcOps<Dc>::add(a1, a2), a3));
    }
    for (int c = ml; c < cn && c0 + c < I.Gb; c += 32) tot = DcOps<Dc>::add(tot, s_pg[tl][c]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot = DcOps<Dc>::add(tot, DcOps<Dc>::shfl_down(tot, o));
  if (ml == 0 && t < I.T)
    s_mu[tl] = DcOps<Dc>::mul(DcOps<Dc>::add(tot, DcOps<Dc>::neg(lt)), DcOps<Dc>::inv_n(I));
  __syncthreads();
  if (out) {
    Dc f = DcOps<Dc>::add(acc, DcOps<Dc>::neg(cl));
    f = DcOps<Dc>::add(f, DcOps<Dc>::neg(DcOps<Dc>::mul(s_mu[tl], rs)));
    if (xi >= 0) f = DcOps<Dc>::add(f, DcOps<Dc>::from_real(bphi));  // a phase shifter's own flow b
    const Real fr = DcOps<Dc>::to_real(f);
    d.fre[e] = fr;
    d.f32[e] = DcOps<Dc>::to_float(f);
    if (kx >= 0) {
      const long long ek = I.tk0 + (long long)t * I.K + kx;
      d.fk[ek] = fr;
      d.fk32[ek] = DcOps<Dc>::to_float(f);
    }
  }
  pold_share(d, I, t0, sub, x);  // after the loads above: its stores would otherwise hold them back
}

// Base DC flows in the sparse mode, from the angles theta' = Yhat^-1 p_inj solved by the sparse
// factor (0 at the reference bus): f[t,m] = y_m (theta'_f - theta'_o) - mu_t (PTDF 1)_m, the last
// term being the uniform slack (Sec. II-E) with mu_t the mean injection.
template <typename Real, typename Dc>
__device__ void s1_sdcf(const Dev<Real, Dc> &d, const Inst &I, int tc, int sub, const Real *__restrict__ x) {
  const int t0 = tc * DCF_TC, m0 = sub * DCF_BM;
  const int t = t0 + (threadIdx.x >> 5), m = m0 + (threadIdx.x & 31);
  pold_share(d, I, t0, sub, x);
  const bool on = t < I.T && m < I.M;
  const int2 ft = d.br_end[I.br0 + (on ? m : 0)];
  const int pf = d.bus_pos[ft.x], po = d.bus_pos[ft.y];
  const Dc y = d.ydc[I.br0 + (on ? m : 0)], rs = d.rsum[I.br0 + (on ? m : 0)];
  pdl_wait();
  if (!on) return;
  Dc a = pf >= 0 ? d.sp_th[(long long)pf * I.T + t] : DcOps<Dc>::zero();
  if (po >= 0) a = DcOps<Dc>::add(a, DcOps<Dc>::neg(d.sp_th[(long long)po * I.T + t]));
  Dc f = DcOps<Dc>::mul(y, a);
  f = DcOps<Dc>::add(f, DcOps<Dc>::neg(DcOps<Dc>::mul(d.sp_mu[t], rs)));
  const int xi = d.br_xf[I.br0 + m];  // a phase shifter's own flow b adds to the monitored flow
  if (xi >= 0)
    f = DcOps<Dc>::add(f, DcOps<Dc>::from_real(d.br_b[I.br0 + m] * x[I.xtau0 + (long long)(I.T + t) * I.X + xi]));
  const long long e = I.tm0 + (long long)t * I.M + m;
  const Real fr = DcOps<Dc>::to_real(f);
  d.fre[e] = fr;
  d.f32[e] = DcOps<Dc>::to_float(f);
  const int kx = d.br_kidx[I.br0 + m];
  if (kx >= 0) {
    const long long ek = I.tk0 + (long long)t * I.K + kx;
    d.fk[ek] = fr;
    d.fk32[ek] = DcOps<Dc>::to_float(f);
  }
}

// Bus balance (Example 4): P_it = load + sum of end flows - sum of generation, as a
// warp-segmented reduction over the bus's CSR entries (each branch end's flow computed in place
// from v, theta: the balance does not wait for the branch role); soft-abs penalty and its derivative.
template <typename Real, typename Dc>
__device__ void s1_bus(const Dev<Real, Dc> &d, const Inst &I, int t, int sub, const Real *__restrict__ x,
                       Obj3<Dc> &acc, const HP<Real> hp) {
  const int pk = sub * PACKS_PER_BLOCK + (threadIdx.x >> 5);
  if (pk >= I.n_bal_pack) return;  // whole warp
  const int e = I.bal0 + pk * PACK + (threadIdx.x & 31);
  const int code = d.bal_code[e], row = d.bal_row[e];
  const int kind = code & 3, id = code >> 2;
  const long long ti = I.tb0 + (long long)t * I.n + (row >= 0 ? row : 0);
  Real P = 0, Q = 0;
  if (kind <= 1) {
    Real pf, qf, pt, qt;
    pi_flow(d, I, t, I.br0 + id, x, pf, qf, pt, qt);
    P = kind == 0 ? pf : pt;
    Q = kind == 0 ? qf : qt;
  } else if (kind == 2) {  // a producer supplies (-), a consumer draws (+)
    const Real sg = d.gen_sgn[I.gen0 + id];
    const Real *p = x + I.x0 + 2LL * I.T * I.n + (long long)t * I.G + id;
    P = -sg * p[0];
    Q = -sg * p[(long long)I.T * I.G];
  }
  if (seg_sum2(row, P, Q) && row >= 0) {
    P += d.load_p[ti];
    Q += d.load_q[ti];
    Real vp, dp, vq, dq;
    soft_abs(P, hp.eps, vp, dp);
    soft_abs(Q, hp.eps, vq, dq);
    const Real dtw = d.dt[I.tp0 + t];
    const Real wp = dtw * d.c_p * hp.beta, wq = dtw * d.c_q * hp.beta;
    d.dP[ti] = wp * dp;
    d.dQ[ti] = wq * dq;
    acc.v[0] = DcOps<Dc>::from_real(wp * vp);
    acc.v[1] = DcOps<Dc>::from_real(wq * vq);
  }
}

template <typename Real, typename Dc>
__global__ void __launch_bounds__(NTHR) k_s1(const __grid_constant__ Dev<Real, Dc> d,
                                             const __grid_constant__ InstTab tab, const __grid_constant__ Spans S,
                                             const Real *__restrict__ x, int slot0) {
  const Where w = locate(S);
  const Inst &I = tab.I[tab.n_inst == 1 ? 0 : w.inst];  // one instance: no wait on the span search
  const int slot = d.slot_map[slot0 + blockIdx.x];  // issued first: it is not needed until the end
  Obj3<Dc> acc = obj3<Dc>(-1);
  if (w.role == R_DCF) {
    s1_dcf(d, I, w.t, w.sub, x);
  } else if (w.role == R_SDCF) {
    s1_sdcf(d, I, w.t, w.sub, x);
  } else if (w.role == R_BRANCH) {
    acc.id[0] = T_ZS;
    s1_branch(d, I, w.t, w.sub, x, acc, hparams(d));
  } else if (w.role == R_BUS) {
    acc.id[0] = T_ZP;
    acc.id[1] = T_ZQ;
    s1_bus(d, I, w.t, w.sub, x, acc, hparams(d));
  } else {
    acc.id[0] = T_ZRZ;
    s1_zone(d, I, w.t, w.sub, x, acc, hparams(d));
  }
  write_obj(d.objp, slot, acc);
}

// ---------------------------------------------------------------------------------------------
// stage 2
// ---------------------------------------------------------------------------------------------

// Bus balance (Example 4) in stage 2 (the FP64 path, and the mixed path of larger plans): the same
// sums as s1_bus from the flows that stage 1 stored (recomputing them would cost the FP64 path its
// slow sincos a second time).  A block covers I.bus_tc consecutive periods of its CSR packs (period
// chunk tc), its objective partials summed over them in period order.
template <typename Real, typename Dc>
__device__ void s2_bus(const Dev<Real, Dc> &d, const Inst &I, int tc, int sub, const Real *__restrict__ x,
                       Obj3<Dc> &acc, const HP<Real> hp) {
  const int pk = sub * PACKS_PER_BLOCK + (threadIdx.x >> 5);
  if (pk >= I.n_bal_pack) return;  // whole warp
  const int e = I.bal0 + pk * PACK + (threadIdx.x & 31);
  const int code = d.bal_code[e], row = d.bal_row[e];
  const int kind = code & 3, id = code >> 2;
  const int ta = tc * I.bus_tc, tz = min(I.T, ta + I.bus_tc);
  // data no earlier stage writes first (loads, weights, the device's role), then wait for stage 1
  const Real sg = kind == 2 ? d.gen_sgn[I.gen0 + id] : Real(1);
  const long long ti0 = I.tb0 + (long long)ta * I.n + (row >= 0 ? row : 0);
  Real lp = d.load_p[ti0], lq = d.load_q[ti0];
  pdl_wait();
  Dc zp = DcOps<Dc>::zero(), zq = DcOps<Dc>::zero();
  for (int t = ta; t < tz; ++t) {
    const long long ti = I.tb0 + (long long)t * I.n + (row >= 0 ? row : 0);
    if (t > ta) {
      lp = d.load_p[ti];
      lq = d.load_q[ti];
    }
    const Real dtw = d.dt[I.tp0 + t];
    Real P = 0, Q = 0;
    const long long tm = I.tm0 + (long long)t * I.M + id;
    if (kind == 0) {
      P = d.pf[tm];
      Q = d.qf[tm];
    } else if (kind == 1) {
      P = d.pt[tm];
      Q = d.qt[tm];
    } else if (kind == 2) {  // a producer supplies (-), a consumer draws (+)
      const Real *p = x + I.x0 + 2LL * I.T * I.n + (long long)t * I.G + id;
      P = -sg * p[0];
      Q = -sg * p[(long long)I.T * I.G];
    }
    if (seg_sum2(row, P, Q) && row >= 0) {
      P += lp;
      Q += lq;
      Real vp, dp, vq, dq;
      soft_abs(P, hp.eps, vp, dp);
      soft_abs(Q, hp.eps, vq, dq);
      const Real wp = dtw * d.c_p * hp.beta, wq = dtw * d.c_q * hp.beta;
      d.dP[ti] = wp * dp;
      d.dQ[ti] = wq * dq;
      zp = DcOps<Dc>::add(zp, DcOps<Dc>::from_real(wp * vp));
      zq = DcOps<Dc>::add(zq, DcOps<Dc>::from_real(wq * vq));
    }
  }
  acc.v[0] = zp;
  acc.v[1] = zq;
}

// Four consecutive entries of the line-outage block (row stride padded to a multiple of 4, so
// the group is one aligned vector load) as floats.
__device__ __forceinline__ void lodf_load4(const void *base, long long idx, int dtype, float (&v)[4]) {
  if (dtype == QG_LODF_BF16) {
    const uint2 u = *reinterpret_cast<const uint2 *>(static_cast<const __nv_bfloat16 *>(base) + idx);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&u.x), b = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
    v[0] = __low2float(a); v[1] = __high2float(a); v[2] = __low2float(b); v[3] = __high2float(b);
  } else if (dtype == QG_LODF_BF16X2) {
    const uint4 u = *reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat162 *>(base) + idx);
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[j]);
      v[j] = __low2float(h) + __high2float(h);
    }
  } else {
    const float4 f = *reinterpret_cast<const float4 *>(static_cast<const float *>(base) + idx);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  }
}

template <typename Real>
__host__ __device__ constexpr int ctg_tch() { return 8; }

// Clearance of a monitored branch in one period for the bound test of the contingency screen: a
// value r <= sqrt(-(qmax2 - s_ctg^2)) (1 - 2^-20) - |f_m|, every step rounded down, or -1 where that
// margin is not at least 2^-40 (no clearance; NaN inputs included).
__device__ __forceinline__ float clear_margin(float f, float qs) {
  const float r = __fsub_rd(__fmul_rd(__fsqrt_rd(-qs), 1.f - 0x1p-20f), fabsf(f));
  return r >= 0x1p-40f ? r : -1.f;
}

// The screen's q-term of a monitored branch in one period, qmax2 - s_ctg^2 in FP32; the FP64 path adds
// the part of its margin that covers the roundings of that difference (the part that covers F is
// added per period in the screen).
template <typename Real>
__device__ __forceinline__ float ctg_qs(Real q2, Real s2) {
  if constexpr (sizeof(Real) == 8) return (float)((q2 - s2) + 0x1p-22 * (fabs(q2 - s2) + s2));
  else return (float)(q2 - s2);
}

// Bound test of one thread's 4 rows over a chunk: Lmax fc < r for each row, with Lmax the rows' largest
// |L| over the thread's 16-outage group, fc that group's largest |f_k| over the chunk and r the rows'
// smallest clearance (all finite, so no NaN can arise).
__device__ __forceinline__ bool bound_clear(float4 lm, float4 rm, float fc) {
  float a0, a1, a2, a3;
  unpack2(fma2(pack2(-lm.x, -lm.y), pack2(fc, fc), pack2(rm.x, rm.y)), a0, a1);
  unpack2(fma2(pack2(-lm.z, -lm.w), pack2(fc, fc), pack2(rm.z, rm.w)), a2, a3);
  return fminf(fmin3(a0, a1, a2), a3) > 0.f;
}

constexpr int CT_TBATCH = 12;  // tiles per batch of bound tests on the on-demand path

// Clearance minima for the on-demand contingency path: for every instance that takes it, chunk
// q = tci NCH + ch (periods [tci ctg_tb + 8 ch, +8) of period range tci) and monitored branch m, the
// smallest clear_margin of the branch over the chunk's periods (FLT_MAX on the pad rows of the last
// 64-row tile), from the FP32 values the stage-2 screen reads.  Once per evaluation, instead of once
// per outage tile.
template <typename Real, typename Dc>
__global__ void __launch_bounds__(NTHR) k_ctg_margin(const __grid_constant__ Dev<Real, Dc> d,
                                                     const __grid_constant__ InstTab tab) {
  pdl_wait();
  for (int b = 0; b < tab.n_inst; ++b) {
    const Inst &I = tab.I[b];
    if (!I.ctg_lazy || I.n_kt == 0) continue;
    const int rows = I.n_mt * CT_BM, nchm = (I.ctg_tb + 7) / 8;
    const long long n = (long long)I.ctg_ntc * nchm * rows;
    for (long long e = blockIdx.x * (long long)NTHR + threadIdx.x; e < n; e += (long long)gridDim.x * NTHR) {
      const int q = (int)(e / rows), m = (int)(e % rows);
      const int tci = q / nchm, ch = q % nchm;
      const int tb0 = tci * I.ctg_tb, TB = min(I.ctg_tb, I.T - tb0);
      const int ta = tb0 + ch * 8, tz = tb0 + min(TB, ch * 8 + 8);
      float r = FLT_MAX;
      if (m < I.M && ta < tz) {
        // the chunk's loads all in flight at once: periods past its end repeat its last one
        const Real s2 = d.br_s2ctg[I.br0 + m];
        float f[8];
        Real q2[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long idx = I.tm0 + (long long)min(ta + j, tz - 1) * I.M + m;
          f[j] = d.f32[idx];
          q2[j] = d.qm2[idx];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) r = fminf(r, clear_margin(f[j], ctg_qs<Real>(q2[j], s2)));
      }
      d.ctg_rmin[I.rm0 + e] = r;
    }
  }
}

// Contingency block (Sec. II-E, Eqs. rank_correct, sfr_pen-zctg) for outages [k0, k0 + 64), the
// monitored-branch tiles of one group (64 branches each) and one chunk of periods:
//   F[t,m,k] = f[t,m] + L[m,k] f[t,k],   s = sqrt(F^2 + qmax2[t,m]),
//   z += w sigma_s(s - s_ctg_m),  dz/dF = w sigma' F / s.
// Thread (row quad rq, column quad cq) holds a 4 x 4 piece of the line-outage tile in registers,
// as pairs of rows per column; per period it reads f, qmax2 - s_ctg^2 of its rows and f_k of its
// columns (stored twice, as the pair {f_k, f_k}) as four 128-bit shared loads and screens its 16
// elements in FP32: two paired FMAs per two elements and a three-input max tree; an element can
// only be overloaded if F^2 + qmax2 - s_ctg^2 > 0.  The FP64 path recomputes candidates exactly
// from the FP64 block; its screen adds a margin derived from a bound on the FP32 errors, so every
// element whose FP64 value is over the limit is a candidate (the bound is at the screen's margin
// below).  Pads and the outaged branch itself carry L = NaN, which the max ignores and every
// compare rejects.
//
// Bound test (I.ctg_bound): before that screen, each warp bounds its 8 rows x 64 outages over a
// chunk of 8 periods at once.  With Lmax the largest |L| of a row over the 16 outages of a thread's
// column group (Dev::lmax, static), fc the largest |f_k| of that group over the chunk and r the
// smallest clearance of the row over the chunk (clear_margin), Lmax fc < r implies, for every
// element, |F32| <= (|L||f_k| + |f_m|)(1 + 2^-24) < sqrt(s_ctg^2 - qmax2) (1 - 2^-20)(1 + 2^-24),
// so the screen's value F32^2 + qmax2 - s_ctg^2 is negative by at least 2^-19 (s_ctg^2 - qmax2)
// (1 - 2^-23): no element is a candidate on either path (the FP64 path's margin adds at most
// 2^-21 (1 + 2^-20) of that), and the warp skips the chunk.  The classification, and so every
// result, is bitwise that of the element screen alone.  The eager path stages each tile's rows
// (flows, q-terms and their clearances), loads every warp's piece of the line-outage tile and tests
// per chunk.  The on-demand path (large plans) takes the clearances per chunk from k_ctg_margin
// (computed once per evaluation rather than once per outage tile), tests every (tile, chunk) of a
// batch of up to CT_TBATCH tiles at once, and stages, loads and screens only the tiles and chunks
// where some warp of the block fails; a warp loads its piece of a tile only if it fails there.
//
// Only warps with a candidate take the exact path and write partial sums (the buffers are zeroed
// per chunk of periods): row sums (dz/df_m, dz/dqmax2_m) by shuffles across the 16 column quads,
// flushed to the partials pm, pq per outage tile; column sums (dz/df_k through L[m,k]) across the
// block's row quads through shared memory, accumulated over the group's tiles and written to pk per
// group; a chunk in which no warp of the block had a candidate skips the flush.  The soft-ReLU
// floor eps of every non-violating element is added in closed form by the final reduction.  MODE
// (Inst::ctg_bound / ctg_lazy, the same for every instance of a plan), compiled apart so that each
// keeps its registers: 0 no bound test, 1 the eager path, 2 the on-demand path.
template <typename Real, typename Dc, int MODE>
__device__ void s2_ctg(const Dev<Real, Dc> &d, const Inst &I, int sub, Obj3<Dc> &acc, const HP<Real> hp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool F64 = sizeof(Real) == 8;
  constexpr int TCH = ctg_tch<Real>();
  static_assert(NTHR == 4 * CT_BM && CT_BM == CT_BK, "staging maps a thread to one row and every fourth chunk");
  const int T = I.T, TBM = I.ctg_tb;
  const int NCHM = (TBM + TCH - 1) / TCH;  // chunks of the longest period range
  // the period chunks of one (group, outage tile) are adjacent blocks: they run together and read
  // the same line-outage rows, the later ones from L2
  const int tci = sub % I.ctg_ntc, rem = sub / I.ctg_ntc, mg = rem / I.n_kt, kt = rem % I.n_kt;
  const int t0 = tci * TBM, TB = min(TBM, T - t0), nch = (TB + TCH - 1) / TCH;
  const int k0 = kt * CT_BK;
  const int mt0 = mg * I.ctg_mg, mt1 = min(I.n_mt, mt0 + I.ctg_mg);
  float *s_fm = reinterpret_cast<float *>(smem_raw);  // [TB][BM] base flow of the monitored branch
  float *s_qs = s_fm + TBM * CT_BM;                   // [TB][BM] qmax2 - s_ctg^2 (+ margin on the FP64 path)
  float *s_fk = s_qs + TBM * CT_BM;                   // [TB][BK][2] base flow of the outaged branch, twice
  float *s_rmin = s_fk + 2 * TBM * CT_BK;             // [NCH][BM] eager bound test: smallest clearance of the row over the chunk
  float *s_fkc = s_rmin + NCHM * CT_BM;               // [NCH][4] largest |f_k| of a 16-outage group over the chunk
  constexpr bool lazy = MODE == 2, bound = MODE != 0;
  float *s_lmb = s_fkc + 4 * NCHM;                    // on-demand path: [TBATCH][4][BM] Lmax of the batch's tiles
  float *s_rmb = s_lmb + (lazy ? CT_TBATCH * 4 * CT_BM : 0);  // on-demand path: [TBATCH][NCH][BM] clearance minima
  Real *s_s2 = reinterpret_cast<Real *>(s_rmb + (lazy ? CT_TBATCH * NCHM * CT_BM : 0));  // [2][BM] s_ctg^2, then s_ctg
  Real *s_gm = s_s2 + 2 * CT_BM;                      // [TCH][BM]
  Real *s_gq = s_gm + TCH * CT_BM;                    // [TCH][BM]
  Real *s_gk = s_gq + TCH * CT_BM;                    // [TCH][8][BK]
  Real *s_ga = s_gk + TCH * 8 * CT_BK;                // [TB][BK] column sums over the group
  Real *s_f64m = s_ga + TBM * CT_BK;                  // [TB][BM] (FP64 path only)
  Real *s_f64k = s_f64m + (F64 ? TBM * CT_BM : 0);    // [TB][BK] (FP64 path only)
  Real *s_gz = s_f64k + (F64 ? TBM * CT_BK : 0);      // [TCH][8][BK] score column sums (screening only)
  Real *s_za = s_gz + (d.score ? TCH * 8 * CT_BK : 0);  // [TB][BK] scores over the group (screening only)
  const bool score = d.score != 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rq = threadIdx.x >> 4, cq = threadIdx.x & 15;
  const int kc = k0 + cq * 4;  // first of this thread's four outages
  const int sc = threadIdx.x & (CT_BM - 1), sp = threadIdx.x >> 6;  // staging: row / column sc, chunks sp, sp + 4, ...
  __shared__ int s_hit[ctg_tch<Real>()];  // per period of the chunk: some row of the tile has a partial
  __shared__ int s_cand[2];               // per chunk (alternating): some warp of the block had a candidate
  __shared__ int s_fail[CT_TBATCH][8];    // on-demand path: per tile of the batch and warp, the chunks failing the bound test
  __shared__ int s_anyf[CT_TBATCH];       // on-demand path: their union over the block's warps
  if (threadIdx.x < TCH) s_hit[threadIdx.x] = 0;
  if (threadIdx.x < 2) s_cand[threadIdx.x] = 0;
  for (int e = threadIdx.x; e < TCH * CT_BM; e += NTHR) s_gm[e] = s_gq[e] = 0;
  for (int e = threadIdx.x; e < TCH * 8 * CT_BK; e += NTHR) s_gk[e] = 0;
  if (score)
    for (int e = threadIdx.x; e < TCH * 8 * CT_BK; e += NTHR) s_gz[e] = 0;
  Real obj = 0;
  const Real eps = hp.eps;
  int cpar = 0;  // chunk parity (s_cand slot)
  // first tile: the outage columns' data (f_k twice, the FP64 copy, zeroed column sums) and the
  // largest |f_k| per 16-outage group and chunk, for column sc over chunks sp, sp + 4, ...
  // (with the bound test; without it the first tile's row staging below does the same per entry)
  auto stage_k = [&]() {
    for (int ch = sp; ch < nch; ch += 4) {
      const int k = k0 + sc;
      float fkm = 0.f;
#pragma unroll
      for (int j = 0; j < TCH; ++j) {
        const int tt = ch * TCH + j;
        if (tt >= TB) break;
        float f = 0.f;
        Real f64 = 0;
        if (k < I.K) {
          const long long idx = I.tk0 + (long long)(t0 + tt) * I.K + k;
          f = d.fk32[idx];
          if (F64) f64 = d.fk[idx];
        }
        *reinterpret_cast<float2 *>(s_fk + 2 * (tt * CT_BK + sc)) = make_float2(f, f);
        if (F64) s_f64k[tt * CT_BK + sc] = f64;
        s_ga[tt * CT_BK + sc] = 0;
        if (score) s_za[tt * CT_BK + sc] = 0;
        fkm = fmaxf(fkm, fabsf(f));  // a NaN flow is ignored: its elements are no candidates either
      }
      // over the 16 outages of the group (16 consecutive lanes); finite, so that the bound test
      // never forms 0 x infinity
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) fkm = fmaxf(fkm, __shfl_xor_sync(0xffffffffu, fkm, o));
      if ((sc & 15) == 0) s_fkc[ch * 4 + (sc >> 4)] = fminf(fkm, FLT_MAX);
    }
  };
  const int rows = I.n_mt * CT_BM;
  // tiles in batches: on the on-demand path, the bound tests of a batch of up to CT_TBATCH tiles come
  // first; the eager path takes all of the group's tiles as one batch and tests per chunk
  for (int mb = mt0; mb < mt1; mb += lazy ? CT_TBATCH : max(1, mt1 - mt0)) {
    const int me = lazy ? min(mt1, mb + CT_TBATCH) : mt1;
    if (lazy) {
      // the batch's test inputs: Lmax (static, before the wait) and the clearance minima of
      // k_ctg_margin
      for (int e = threadIdx.x; e < (me - mb) * 4 * CT_BM; e += NTHR) {
        const int bt = e / (4 * CT_BM), g = (e / CT_BM) & 3, r = e % CT_BM;
        s_lmb[e] = d.lmax[I.lm0 + (long long)(kt * 4 + g) * rows + (mb + bt) * CT_BM + r];
      }
      if (threadIdx.x < CT_TBATCH) s_anyf[threadIdx.x] = 0;
      if (mb == mt0) {
        pdl_wait();
        stage_k();
      }
      for (int e = threadIdx.x; e < (me - mb) * nch * CT_BM; e += NTHR) {
        const int bt = e / (nch * CT_BM), ch = (e / CT_BM) % nch, r = e % CT_BM;
        s_rmb[(bt * NCHM + ch) * CT_BM + r] = d.ctg_rmin[I.rm0 + (long long)(tci * NCHM + ch) * rows + (mb + bt) * CT_BM + r];
      }
      __syncthreads();
      // per tile of the batch and warp: the chunks whose bound test fails
      for (int bt = 0; bt < me - mb; ++bt) {
        const float4 lm = *reinterpret_cast<const float4 *>(s_lmb + (bt * 4 + (cq >> 2)) * CT_BM + rq * 4);
        int fail = 0;
        for (int ch = 0; ch < nch; ++ch) {
          const float4 rm = *reinterpret_cast<const float4 *>(s_rmb + (bt * NCHM + ch) * CT_BM + rq * 4);
          if (!__all_sync(0xffffffffu, bound_clear(lm, rm, s_fkc[ch * 4 + (cq >> 2)]))) fail |= 1 << ch;
        }
        if (lane == 0) {
          s_fail[bt][wid] = fail;
          if (fail) atomicOr(&s_anyf[bt], fail);  // an OR: the same in any order
        }
      }
      __syncthreads();
    }
    for (int mt = mb; mt < me; ++mt) {
      const int m0 = mt * CT_BM;
      // on-demand path: chunks where this warp / some warp of the block must screen (s_fail, s_anyf)
      const int bt = mt - mb;
      if (lazy && !s_anyf[bt]) {  // every warp passes every chunk: no partial of this tile, zero flags
        if (threadIdx.x < TB) d.pmf[I.pf0 + ((long long)kt * T + t0 + threadIdx.x) * I.n_mt + mt] = 0;
        continue;
      }
      // this thread's piece of the line-outage tile, as row pairs (FP64 path: the largest |L| of each
      // row over its four columns; a NaN column is ignored); static data, which the eager paths load
      // before any wait and the on-demand path only in failing warps
      f32x2 Lp[2][4];  // {L[2h][j], L[2h + 1][j]}
      float Lrow[4];
      auto load_L = [&]() {
        float L[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m = m0 + rq * 4 + i;
          if (m < I.M && kc < I.Kp) {
            lodf_load4(d.lodf, I.l0 + (long long)m * I.Kp + kc, d.lodf_dtype, L[i]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) L[i][j] = f_nan();
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 4; ++j) Lp[h][j] = pack2(L[2 * h][j], L[2 * h + 1][j]);
        if (F64) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            Lrow[i] = fmaxf(fmaxf(fabsf(L[i][0]), fabsf(L[i][1])), fmaxf(fabsf(L[i][2]), fabsf(L[i][3])));
        }
      };
      bool have_L = false;
      if (!lazy) {
        load_L();
        have_L = true;
      } else if (s_fail[bt][wid]) {  // the failing warps' loads overlap the staging below
        load_L();
        have_L = true;
      }
      const Real s2m = (threadIdx.x < CT_BM && m0 + threadIdx.x < I.M) ? d.br_s2ctg[I.br0 + m0 + threadIdx.x] : Real(0);
      if (threadIdx.x < CT_BM) {
        s_s2[threadIdx.x] = s2m;
        s_s2[CT_BM + threadIdx.x] = dsqrt(s2m);
      }
      if (!lazy && mt == mt0) {
        pdl_wait();
        if (bound) stage_k();
      }
      // the rows' data: flows, q_max^2 - s_ctg^2 and the FP64 flows; on the eager path with the bound
      // test, for row sc over chunks sp, sp + 4, ... with the smallest clearance per chunk (FLT_MAX on
      // pad rows: they never fail the test), else entries e = (period, row) over every thread
      if (MODE != 1) {
        // without the bound test the first tile also stages the outage columns' data here (CT_BK ==
        // CT_BM), so that both loads are in flight together
        const bool with_k = MODE == 0 && mt == mt0;
#pragma unroll 4
        for (int e = threadIdx.x; e < TB * CT_BM; e += NTHR) {
          const int tt = e / CT_BM, c = e % CT_BM, m = m0 + c;
          float f = 0.f, qs = 0.f, fk = 0.f;
          Real f64 = 0, fk64 = 0;
          if (with_k && k0 + c < I.K) {
            const long long idx = I.tk0 + (long long)(t0 + tt) * I.K + k0 + c;
            fk = d.fk32[idx];
            if (F64) fk64 = d.fk[idx];
          }
          if (m < I.M) {
            const long long idx = I.tm0 + (long long)(t0 + tt) * I.M + m;
            f = d.f32[idx];
            qs = ctg_qs<Real>(d.qm2[idx], d.br_s2ctg[I.br0 + m]);
            if (F64) f64 = d.fre[idx];
          }
          s_fm[tt * CT_BM + c] = f;
          s_qs[tt * CT_BM + c] = qs;
          if (F64) s_f64m[tt * CT_BM + c] = f64;
          if (with_k) {
            *reinterpret_cast<float2 *>(s_fk + 2 * (tt * CT_BK + c)) = make_float2(fk, fk);
            if (F64) s_f64k[tt * CT_BK + c] = fk64;
            s_ga[tt * CT_BK + c] = 0;
            if (score) s_za[tt * CT_BK + c] = 0;
          }
        }
      }
      for (int ch = sp; MODE == 1 && ch < nch; ch += 4) {
        const int m = m0 + sc;
        const Real s2 = m < I.M ? d.br_s2ctg[I.br0 + m] : Real(0);
        float rmin = FLT_MAX;
#pragma unroll
        for (int j = 0; j < TCH; ++j) {
          const int tt = ch * TCH + j;
          if (tt >= TB) break;
          float f = 0.f, qs = 0.f;
          Real f64 = 0;
          if (m < I.M) {
            const long long idx = I.tm0 + (long long)(t0 + tt) * I.M + m;
            f = d.f32[idx];
            qs = ctg_qs<Real>(d.qm2[idx], s2);
            if (F64) f64 = d.fre[idx];
            rmin = fminf(rmin, clear_margin(f, qs));
          }
          s_fm[tt * CT_BM + sc] = f;
          s_qs[tt * CT_BM + sc] = qs;
          if (F64) s_f64m[tt * CT_BM + sc] = f64;
        }
        s_rmin[ch * CT_BM + sc] = rmin;
      }
      __syncthreads();
      for (int tc0 = 0, ch = 0; tc0 < TB; tc0 += TCH, ++ch, cpar ^= 1) {
        const int tn = min(TCH, TB - tc0);
        bool skip = false;
        if (lazy) {
          if (!((s_anyf[bt] >> ch) & 1)) {  // no warp screens this chunk (block-uniform): zero flags only
            if (threadIdx.x < tn) d.pmf[I.pf0 + ((long long)kt * T + t0 + tc0 + threadIdx.x) * I.n_mt + mt] = 0;
            continue;
          }
          skip = !((s_fail[bt][wid] >> ch) & 1);
        } else if (bound) {
          // bound test of the warp's 8 rows x 64 outages over the chunk; Lmax of this thread's rows over
          // its column group (static) is reread per chunk from L1, so that no register holds it
          // through the screen
          const float4 lm = __ldg(reinterpret_cast<const float4 *>(d.lmax + I.lm0 + (long long)(kt * 4 + (cq >> 2)) * rows +
                                                                  m0 + rq * 4));
          const float4 rm = *reinterpret_cast<const float4 *>(s_rmin + ch * CT_BM + rq * 4);
          skip = __all_sync(0xffffffffu, bound_clear(lm, rm, s_fkc[ch * 4 + (cq >> 2)]));
        }
        if (!skip && !have_L) {
          load_L();
          have_L = true;
        }
        for (int tt = 0; tt < tn && !skip; ++tt) {
          const int tl = tc0 + tt;
          const float4 fm4 = *reinterpret_cast<const float4 *>(s_fm + tl * CT_BM + rq * 4);
          const float4 qs4 = *reinterpret_cast<const float4 *>(s_qs + tl * CT_BM + rq * 4);
          const float4 fka = *reinterpret_cast<const float4 *>(s_fk + 2 * (tl * CT_BK + cq * 4));
          const float4 fkb = *reinterpret_cast<const float4 *>(s_fk + 2 * (tl * CT_BK + cq * 4) + 4);
          const float fm[4] = {fm4.x, fm4.y, fm4.z, fm4.w};
          float qs[4] = {qs4.x, qs4.y, qs4.z, qs4.w};
          const f32x2 fkd[4] = {pack2(fka.x, fka.y), pack2(fka.z, fka.w), pack2(fkb.x, fkb.y), pack2(fkb.z, fkb.w)};
          if (F64) {
            // the rest of the screen's margin: the FP32 value of F = f_m + L f_k is off by at most
            // 3.0001 u (|f_m| + |L||f_k|) (u = 2^-24; three roundings: L, f_k, f_m to FP32 and the fma),
            // so |F32^2 - F^2| <= 6.0003 u A^2 with A <= Ahat = |f_m| + max|L| max|f_k| over the
            // thread's columns; 2^-21 Ahat^2 = 8 u Ahat^2 covers it and the FP64 rounding of the exact test
            const float fkq = fmaxf(fmaxf(fabsf(fka.x), fabsf(fka.z)), fmaxf(fabsf(fkb.x), fabsf(fkb.z)));
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float ah = __fmaf_rn(Lrow[i], fkq, fabsf(fm[i]));
              qs[i] = __fadd_rn(qs[i], __fmul_rn(__fmul_rn(ah, ah), 0x1p-21f));
            }
          }
          const f32x2 fmp[2] = {pack2(fm[0], fm[1]), pack2(fm[2], fm[3])};
          const f32x2 qsp[2] = {pack2(qs[0], qs[1]), pack2(qs[2], qs[3])};
          // F = fma(L, f_k, f_m), y = fma(F, F, qmax2 - s_ctg^2): two paired FMAs per two rows
          float F[4][4], y[4][4];
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const f32x2 Fh = fma2(Lp[h][j], fkd[j], fmp[h]);
              unpack2(Fh, F[2 * h][j], F[2 * h + 1][j]);
              unpack2(fma2(Fh, Fh, qsp[h]), y[2 * h][j], y[2 * h + 1][j]);
            }
          // the largest of the 16 (NaN operands are ignored), as a three-input max tree of depth 3
          const float a0 = fmax3(y[0][0], y[0][1], y[0][2]), a1 = fmax3(y[0][3], y[1][0], y[1][1]);
          const float a2 = fmax3(y[1][2], y[1][3], y[2][0]), a3 = fmax3(y[2][1], y[2][2], y[2][3]);
          const float a4 = fmax3(y[3][0], y[3][1], y[3][2]);
          const float mx = fmaxf(fmax3(a0, a1, a2), fmax3(a3, a4, y[3][3]));
          // a candidate: F^2 + qmax2 - s_ctg^2 > 0 (mixed path: its classification), or, on the FP64
          // path, >= 0 with the margin (a positive exact sum cannot round to a negative one)
          if (!__any_sync(0xffffffffu, F64 ? mx >= 0.f : mx > 0.f)) continue;
          // a (candidate) post-contingency overload in this warp
          if (lane == 0) s_cand[cpar] = 1;
          const Real w = __ldg(d.dt + I.tp0 + t0 + tl) * d.c_s * hp.beta;
          Real gm[4] = {0, 0, 0, 0}, gq[4] = {0, 0, 0, 0}, gk[4] = {0, 0, 0, 0}, zc[4] = {0, 0, 0, 0};
          if (F64 ? mx >= 0.f : mx > 0.f) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int mm = rq * 4 + i;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (!(F64 ? y[i][j] >= 0.f : y[i][j] > 0.f)) continue;  // NaN (pad, outaged branch) fails too
                const Real q2 = d.qm2[I.tm0 + (long long)(t0 + tl) * I.M + m0 + mm];
                Real Fx, Lx, sv, dd;
                if (F64) {
                  Lx = (Real)d.lodf64[I.l0 + (long long)(m0 + mm) * I.Kp + kc + j];
                  Fx = s_f64m[tl * CT_BM + mm] + Lx * s_f64k[tl * CT_BK + cq * 4 + j];
                  if (Fx * Fx + q2 - s_s2[mm] <= Real(0)) continue;
                  sv = dsqrt(Fx * Fx + q2);
                  Real val, der;
                  soft_relu(sv - s_s2[CT_BM + mm], eps, val, der);
                  obj += w * (val - eps);
                  zc[j] += w * (val - eps);
                  dd = w * der / sv;  // dz/dF = w sigma' F / s
                } else {
                  // mixed path: s = sqrt(F^2 + qmax2) and the soft-ReLU through reciprocal square
                  // roots (a few units in the last place, below the FP32 error of F itself)
                  float l0, l1;
                  unpack2(Lp[i >> 1][j], l0, l1);
                  Lx = (i & 1) ? l1 : l0;
                  Fx = F[i][j];
                  const float a2 = __fmaf_rn(F[i][j], F[i][j], (float)q2);
                  const float ra = rsqrtf(a2);
                  const float u = fmaxf(__fmaf_rn(a2, ra, -(float)s_s2[CT_BM + mm]), 0.f);
                  const float b2 = __fmaf_rn(u, u, (float)(eps * eps));
                  const float rb = rsqrtf(b2);
                  const float val = b2 * rb;  // sqrt(u^2 + eps^2)
                  obj += w * (val - eps);
                  zc[j] += w * (val - eps);
                  dd = w * (u * rb) * ra;  // w sigma'(s - s_ctg) / s
                }
                gm[i] += dd * Fx;
                gk[j] += dd * Fx * Lx;
                gq[i] += Real(0.5) * dd;     // dz/dqmax2 = w sigma' / (2 s)
              }
            }
          }
          // row sums across the 16 column quads of each half-warp, when some row of this warp has an
          // overload (the buffers hold zeros otherwise): a reduce-scatter of the thread's 8 values
          // (gm, gq of its 4 rows); each exchange halves what a lane holds, so after three of them
          // lane pair (2v, 2v + 1) of the half-warp holds value v, and a fourth completes its sum
          if (__any_sync(0xffffffffu, (gq[0] != Real(0)) | (gq[1] != Real(0)) | (gq[2] != Real(0)) | (gq[3] != Real(0)))) {
            const bool h8 = cq & 8, h4 = cq & 4, h2 = cq & 2;
            Real r4[4], r2[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // values 0-3: gm, 4-7: gq; lanes with bit 3 keep 4-7
              const Real lo = gm[q], hi = gq[q];
              r4[q] = (h8 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h8 ? lo : hi, 8);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)  // bit 2 keeps entries 2-3 of the four
              r2[q] = (h4 ? r4[q + 2] : r4[q]) + __shfl_xor_sync(0xffffffffu, h4 ? r4[q] : r4[q + 2], 4);
            Real r1 = (h2 ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? r2[0] : r2[1], 2);
            r1 += __shfl_xor_sync(0xffffffffu, r1, 1);
            if (!(cq & 1)) {  // value v = 4 h8 + 2 h4 + h2: row v & 3 of gm (v < 4) or gq
              const int v = cq >> 1;
              ((v & 4) ? s_gq : s_gm)[tt * CT_BM + rq * 4 + (v & 3)] = r1;
            }
            if (lane == 0) s_hit[tt] = 1;
          }
          // column sums across the two row quads of this warp, then per warp through shared memory
#pragma unroll
          for (int j = 0; j < 4; ++j) gk[j] += __shfl_xor_sync(0xffffffffu, gk[j], 16);
          if (lane < 16)
#pragma unroll
            for (int j = 0; j < 4; ++j) s_gk[(tt * 8 + wid) * CT_BK + cq * 4 + j] = gk[j];
          if (score) {  // per-outage scores for the screening list, the same way as the column sums
#pragma unroll
            for (int j = 0; j < 4; ++j) zc[j] += __shfl_xor_sync(0xffffffffu, zc[j], 16);
            if (lane < 16)
#pragma unroll
              for (int j = 0; j < 4; ++j) s_gz[(tt * 8 + wid) * CT_BK + cq * 4 + j] = zc[j];
          }
        }
        __syncthreads();
        const long long pfq = I.pf0 + ((long long)kt * T + t0 + tc0) * I.n_mt + mt;
        if (!s_cand[cpar]) {  // no candidate in the block: no partials, the buffers still hold zeros
          if (threadIdx.x < tn) d.pmf[pfq + (long long)threadIdx.x * I.n_mt] = 0;
          continue;
        }
        // flush the chunk: the row partials of periods with an overload (and their flags); each
        // entry is read and re-zeroed by the same thread
        for (int e = threadIdx.x; e < tn * CT_BM; e += NTHR) {
          const int tt = e / CT_BM, c = e % CT_BM, m = m0 + c;
          if (!s_hit[tt]) continue;
          if (m < I.M) {
            const long long q = I.pm0 + ((long long)kt * T + t0 + tc0 + tt) * I.M + m;
            d.pm[q] = s_gm[e];
            d.pq[q] = s_gq[e];
          }
          s_gm[e] = s_gq[e] = 0;
        }
        if (threadIdx.x < tn) d.pmf[pfq + (long long)threadIdx.x * I.n_mt] = (unsigned char)s_hit[threadIdx.x];
        for (int e = threadIdx.x; e < tn * CT_BK; e += NTHR) {
          const int tt = e / CT_BK, c = e % CT_BK;
          Real sum = s_ga[(tc0 + tt) * CT_BK + c];
#pragma unroll
          for (int ww = 0; ww < 8; ++ww) {
            Real &g = s_gk[(tt * 8 + ww) * CT_BK + c];
            sum += g;
            g = 0;
          }
          s_ga[(tc0 + tt) * CT_BK + c] = sum;
          if (score) {
            Real zsum = s_za[(tc0 + tt) * CT_BK + c];
#pragma unroll
            for (int ww = 0; ww < 8; ++ww) {
              Real &zz = s_gz[(tt * 8 + ww) * CT_BK + c];
              zsum += zz;
              zz = 0;
            }
            s_za[(tc0 + tt) * CT_BK + c] = zsum;
          }
        }
        __syncthreads();
        if (threadIdx.x < TCH) s_hit[threadIdx.x] = 0;
        if (threadIdx.x == 0) s_cand[cpar] = 0;
        __syncthreads();
      }
    }
  }
  for (int e = threadIdx.x; e < TB * CT_BK; e += NTHR) {
    const int tt = e / CT_BK, c = e % CT_BK, k = k0 + c;
    if (k < I.K) {
      const long long q = I.pk0 + ((long long)mg * T + t0 + tt) * I.K + k;
      d.pk[q] = s_ga[tt * CT_BK + c];
      if (score) d.pz[q] = s_za[tt * CT_BK + c];
    }
  }
  acc.v[0] = DcOps<Dc>::from_real(obj);
}

template <typename Real, typename Dc, int MODE>
__global__ void __launch_bounds__(NTHR, sizeof(Real) == 4 ? 3 : 2) k_s2(const __grid_constant__ Dev<Real, Dc> d,
                                             const __grid_constant__ InstTab tab, const __grid_constant__ Spans S,
                                             const Real *__restrict__ x, int slot0) {
  const Where w = locate(S);
  const Inst &I = tab.I[tab.n_inst == 1 ? 0 : w.inst];  // one instance: no wait on the span search
  Obj3<Dc> acc = obj3<Dc>(-1);
  if (w.role == R_BUS) {  // FP64 path
    acc.id[0] = T_ZP;
    acc.id[1] = T_ZQ;
    s2_bus(d, I, w.t, w.sub, x, acc, hparams(d));  // waits after its static loads
  } else {
    acc.id[0] = T_ZCTG;
    s2_ctg<Real, Dc, MODE>(d, I, w.sub, acc, hparams(d));
  }
  write_obj(d.objp, d.slot_map[slot0 + blockIdx.x], acc);
}

// ---------------------------------------------------------------------------------------------
// stage 3: dz/df per branch (sum of the contingency partials), branch-end adjoints
// ---------------------------------------------------------------------------------------------

// Loads through L2 only (no L1 copy that another block's writes could leave stale).
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ df32 ldcg(const df32 *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));  // slots are 8-byte aligned
  return df32{v.x, v.y};
}

// Deterministic block sum of N_TERMS values per thread; the result is valid in thread 0.
template <typename Dc>
__device__ void block_sum_terms(Dc (&a)[N_TERMS]) {
  __shared__ Dc red[NTHR / 32][N_TERMS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N_TERMS; ++k)
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) a[k] = DcOps<Dc>::add(a[k], DcOps<Dc>::shfl_down(a[k], q));
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N_TERMS; ++k) red[wid][k] = a[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < N_TERMS; ++k) {
      Dc v = red[0][k];
#pragma unroll
      for (int q = 1; q < NTHR / 32; ++q) v = DcOps<Dc>::add(v, red[q][k]);
      a[k] = v;
    }
}

// Objective reduction, level 1, run by the fold blocks of stage 3 (off the critical path of the
// last stage): fold block r of an instance sums its stage-1/2 slots [r NTHR, (r + 1) NTHR) (instance-
// major, contiguous) into its fold slot.  Stage 3 waited on stage 2, which waited on stage 1, so
// those slots are complete.
template <typename Real, typename Dc>
__device__ void fold_slots(const Dev<Real, Dc> &d, const Inst &I, int r) {
  Dc a[N_TERMS];
#pragma unroll
  for (int k = 0; k < N_TERMS; ++k) a[k] = DcOps<Dc>::zero();
  const int s = r * NTHR + threadIdx.x;
  if (s < I.obj_n)
#pragma unroll
    for (int k = 0; k < N_TERMS; ++k) a[k] = d.objp[(long long)(I.obj_lo + s) * N_TERMS + k];
  block_sum_terms(a);
  if (threadIdx.x == 0) {
    Dc *dst = d.objp + (long long)(d.n_obj12 + d.n_gen_slots + I.fold_slot0 + r) * N_TERMS;
#pragma unroll
    for (int k = 0; k < N_TERMS; ++k) dst[k] = a[k];
  }
}

template <typename Real, typename Dc, int SPLIT>
__global__ void __launch_bounds__(NTHR, sizeof(Real) == 4 ? 3 : 2) k_s3(const __grid_constant__ Dev<Real, Dc> d,
                                             const __grid_constant__ InstTab tab, const __grid_constant__ Spans S,
                                             const Real *__restrict__ x) {
  const Where w = locate(S);
  const Inst &I = tab.I[tab.n_inst == 1 ? 0 : w.inst];  // one instance: no wait on the span search
  if (w.role == R_OBJ) {  // whole block
    pdl_wait();
    fold_slots(d, I, w.sub);
    return;
  }
  const int t = w.t;
  // SPLIT threads per branch: each sums every SPLIT-th partial, then a fixed-order shuffle
  // tree combines them (the same bits in every thread of the group); the group's first thread
  // loads the branch's flows and adjoints meanwhile and finishes the branch

  const int q = threadIdx.x % SPLIT;
  const int j = w.sub * (NTHR / SPLIT) + threadIdx.x / SPLIT;
  const bool on = j < I.M;
  const int jg = I.br0 + (on ? j : 0);
  // network data first (independent of the earlier stages), then wait
  const int2 ft = d.br_end[jg];
  const int kx = d.br_kidx[jg];
  const Real g = d.br_g[jg], bb = d.br_b[jg], hch = d.br_hch[jg], smax = d.br_smax[jg];
  int xi0 = -1;
  if (I.X > 0) xi0 = d.br_xf[jg];
  pdl_wait();
  const bool lead = on && q == 0;
  const long long e = I.tm0 + (long long)t * I.M + (on ? j : 0);
  // every load of the earlier stages' results is issued before the first store (a store to a
  // possibly aliasing array would keep later loads behind it): end adjoints, flows, voltages
  const long long tb = I.tb0 + (long long)t * I.n;
  Real gpf = 0, gpt = 0, gqf = 0, gqt = 0, pf = 0, qf = 0, pt = 0, qt = 0, vf0 = 1, vo = 1, thf = 0, tho = 0;
  bool qto = false;
  Real tau = Real(1), phi = Real(0);
  if (lead) {
    gpf = d.dP[tb + ft.x];
    gpt = d.dP[tb + ft.y];
    gqf = d.dQ[tb + ft.x];
    gqt = d.dQ[tb + ft.y];
    pf = d.pf[e];
    qf = d.qf[e];
    pt = d.pt[e];
    qt = d.qt[e];
    qto = d.qside[e] != 0;
    const Real *v = x + I.x0 + (long long)t * I.n;
    const Real *th = v + (long long)I.T * I.n;
    vf0 = v[ft.x];
    vo = v[ft.y];
    thf = th[ft.x];
    tho = th[ft.y];
    if (xi0 >= 0) {
      tau = x[I.xtau0 + (long long)t * I.X + xi0];
      phi = x[I.xtau0 + (long long)(I.T + t) * I.X + xi0];
    }
  }
  Real gF = 0, gq2 = 0, gk = 0, zk = 0;
  if (on) {
    // row partials of the outage tiles whose 64-row tile had an overload (flagged by stage 2): few
    // tiles are read unconditionally and selected (no dependent load), many are skipped
    if (I.n_kt <= 16 * SPLIT) {
#pragma unroll 4
      for (int kt = q; kt < I.n_kt; kt += SPLIT) {
        const long long pq = I.pm0 + ((long long)kt * I.T + t) * I.M + j;
        const bool f = d.pmf[I.pf0 + ((long long)kt * I.T + t) * I.n_mt + (j >> 6)] != 0;
        const Real a = d.pm[pq], b = d.pq[pq];
        gF += f ? a : Real(0);
        gq2 += f ? b : Real(0);
      }
    } else {
      for (int kt = q; kt < I.n_kt; kt += SPLIT) {
        if (!d.pmf[I.pf0 + ((long long)kt * I.T + t) * I.n_mt + (j >> 6)]) continue;
        const long long pq = I.pm0 + ((long long)kt * I.T + t) * I.M + j;
        gF += d.pm[pq];
        gq2 += d.pq[pq];
      }
    }
    if (kx >= 0) {
#pragma unroll 8
      for (int mg = q; mg < I.n_mg; mg += SPLIT) gk += d.pk[I.pk0 + ((long long)mg * I.T + t) * I.K + kx];
      if (d.score)
        for (int mg = q; mg < I.n_mg; mg += SPLIT) zk += d.pz[I.pk0 + ((long long)mg * I.T + t) * I.K + kx];
    }
  }
#pragma unroll
#pragma unroll
  for (int o = 1; o < SPLIT; o <<= 1) {
    gF += __shfl_xor_sync(0xffffffffu, gF, o);
    gq2 += __shfl_xor_sync(0xffffffffu, gq2, o);
    gk += __shfl_xor_sync(0xffffffffu, gk, o);
    zk += __shfl_xor_sync(0xffffffffu, zk, o);
  }
  gF += gk;
  if (lead) {
    // adjoints of the four end flows
    const Real sf2 = pf * pf + qf * qf, st2 = pt * pt + qt * qt;
    if (fmax(sf2, st2) > smax * smax) {  // thermal (Example 1)
      const Real sf = dsqrt(sf2), st = dsqrt(st2);
      const bool fr = sf >= st;
      Real val, der;
      const HP<Real> hp = hparams(d);
      soft_relu((fr ? sf : st) - smax, hp.eps, val, der);
      const Real k = d.dt[I.tp0 + t] * d.c_s * hp.beta * der / (fr ? sf : st);
      if (fr) {
        gpf += k * pf;
        gqf += k * qf;
      } else {
        gpt += k * pt;
        gqt += k * qt;
      }
    }
    if (qto) gqt += Real(2) * qt * gq2;  // contingency reactive part, larger-|q| end
    else gqf += Real(2) * qf * gq2;
    const int xi = xi0;
    const Real vf = vf0 / tau;  // vf stands for v_f / tau
    Real sn, cs;
    dsincos(thf - tho - phi, &sn, &cs);
    const Real bc = bb + hch;
    const Real vv = vf * vo;
    const Real A = -g * cs - bb * sn, B = bb * cs - g * sn, C = -g * cs + bb * sn, D = bb * cs + g * sn;
    // adjoint of v_f / tau; d/dv_f = (1/tau) d/d(v_f/tau), d/dtau = -(v_f/tau^2) d/d(v_f/tau)
    const Real au = gpf * (2 * g * vf + A * vo) + gqf * (-2 * bc * vf + B * vo) + gpt * (C * vo) + gqt * (D * vo);
    d.gF[e] = gF;
    if (kx >= 0 && d.score) d.zs[I.tk0 + (long long)t * I.K + kx] = zk;
    d.avf[e] = au / tau;
    if (xi >= 0) d.atx[I.tx0 + (long long)t * I.X + xi] = -au * vf / tau;
    d.avo[e] = gpf * (A * vf) + gqf * (B * vf) + gpt * (2 * g * vo + C * vf) + gqt * (-2 * bc * vo + D * vf);
    d.ad[e] = vv * (gpf * (g * sn - bb * cs) + gqf * (-bb * sn - g * cs) + gpt * (g * sn + bb * cs) +
                    gqt * (-bb * sn + g * cs));
  }
}

// ---------------------------------------------------------------------------------------------
// stage 4: bus gather of branch-end adjoints; adjoint DC products
// ---------------------------------------------------------------------------------------------

template <typename Real>
__device__ __forceinline__ void adam_update(Real &xk, Real gk, Real &mk, Real &vk, Real lo, Real hi, Real b1, Real b2,
                                            Real c1, Real c2, Real lr, Real eps, int paper_eps) {
  mk = b1 * mk + (Real(1) - b1) * gk;
  vk = b2 * vk + (Real(1) - b2) * gk * gk;
  const Real mh = mk * c1, vh = vk * c2;
  const Real num = paper_eps ? mh + eps : mh;
  const Real xn = xk - lr * num / (dsqrt(vh) + eps);
  xk = xn < lo ? lo : (xn > hi ? hi : xn);
}

template <typename Real>
struct AdamCoef {
  Real b1, b2, c1, c2, lr, eps;
  long long step;  // the step counter this update reads (i - 1)
};

// Bias corrections 1 / (1 - beta^i) for the next step i, computed once per block: FP32 through
// expm1 / log1p on the mixed path (1 - beta^i = -expm1(i log1p(beta - 1))); on the FP64 path beta^i
// by the binary square-and-multiply method (Knuth, TAOCP Vol. 2, Sec. 4.6.3): about 2 log2(i)
// multiplications, a few ulp from the correctly rounded power, and far fewer FP64 instructions than
// a general power function.
__device__ __forceinline__ void bias_corr(double b1, double b2, long long step, float &c1, float &c2) {
  const float i = (float)(step + 1);
  c1 = -1.0f / expm1f(i * log1pf((float)b1 - 1.0f));
  c2 = -1.0f / expm1f(i * log1pf((float)b2 - 1.0f));
}
__device__ __forceinline__ void bias_corr(double b1, double b2, long long step, double &c1, double &c2) {
  double p1 = 1.0, p2 = 1.0;
  for (long long i = step + 1; i > 0; i >>= 1) {
    if (i & 1) {
      p1 *= b1;
      p2 *= b2;
    }
    b1 *= b1;
    b2 *= b2;
  }
  c1 = 1.0 / (1.0 - p1);
  c2 = 1.0 / (1.0 - p2);
}

template <typename Real, typename Dc>
__device__ AdamCoef<Real> adam_coef(const Dev<Real, Dc> &d) {
  __shared__ Real sc[3];
  __shared__ long long s_step;
  if (threadIdx.x == 0) {
    const long long step = *d.step + d.step_off;
    bias_corr(d.b1, d.b2, step, sc[0], sc[1]);
    sc[2] = (Real)(d.sched ? d.sched[3 * sched_index(d)] : d.lr);  // step size (Eq. step_size schedule)
    s_step = step;
  }
  __syncthreads();
  return {(Real)d.b1, (Real)d.b2, sc[0], sc[1], sc[2], (Real)d.aeps, s_step};
}

template <typename Real, typename Dc, bool ADAM>
__device__ void s4_bus(const Dev<Real, Dc> &d, const Inst &I, int t, int sub, Real *__restrict__ x,
                       const AdamCoef<Real> &ac) {
  // I.s4p (<= S4_PACKS) consecutive packs per warp: the loads of all of them are issued together
  Real s_x[S4_PACKS][2], s_m[S4_PACKS][2], s_v[S4_PACKS][2], s_lo[S4_PACKS][2], s_hi[S4_PACKS][2];
  int code[S4_PACKS], row[S4_PACKS];
  long long kv[S4_PACKS];
  bool on[S4_PACKS];
  // static CSR entries and (fused Adam) the bus's optimizer state first, then wait for stage 3's
  // branch-end adjoints (no earlier stage of this evaluation writes x, m, v or the box)
#pragma unroll
  for (int u = 0; u < S4_PACKS; ++u) {
    const int pk = (sub * PACKS_PER_BLOCK + (threadIdx.x >> 5)) * I.s4p + u;
    on[u] = u < I.s4p && pk < I.n_adj_pack;
    const int e = I.adj0 + (on[u] ? pk : 0) * PACK + (threadIdx.x & 31);
    code[u] = d.adj_code[e];
    row[u] = on[u] ? d.adj_row[e] : -1;
    kv[u] = I.x0 + (long long)t * I.n + (row[u] >= 0 ? row[u] : 0);
    const long long k2[2] = {kv[u], kv[u] + (long long)I.T * I.n};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      s_x[u][c] = s_m[u][c] = s_v[u][c] = s_lo[u][c] = s_hi[u][c] = Real(0);
      if (ADAM && row[u] >= 0) {
        s_x[u][c] = x[k2[c]];
        s_m[u][c] = d.am[k2[c]];
        s_v[u][c] = d.av[k2[c]];
        s_lo[u][c] = d.lo[k2[c]];
        s_hi[u][c] = d.hi[k2[c]];
      }
    }
  }
  pdl_wait();
  Real gv[S4_PACKS], gth[S4_PACKS];
#pragma unroll
  for (int u = 0; u < S4_PACKS; ++u) {
    const int kind = code[u] & 3;
    gv[u] = gth[u] = Real(0);
    const long long tm = I.tm0 + (long long)t * I.M + (code[u] >> 2);
    if (on[u] && kind == 0) {
      gv[u] = d.avf[tm];
      gth[u] = d.ad[tm];
    } else if (on[u] && kind == 1) {
      gv[u] = d.avo[tm];
      gth[u] = -d.ad[tm];
    }
  }
#pragma unroll
  for (int u = 0; u < S4_PACKS; ++u) {
    if (!on[u]) break;  // whole warp (packs past the end)
    if (seg_sum2(row[u], gv[u], gth[u]) && row[u] >= 0) {
      const long long k2[2] = {kv[u], kv[u] + (long long)I.T * I.n};
      if (ADAM) {
        const Real g2[2] = {gv[u], gth[u]};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          adam_update(s_x[u][c], g2[c], s_m[u][c], s_v[u][c], s_lo[u][c], s_hi[u][c], ac.b1, ac.b2, ac.c1, ac.c2,
                      ac.lr, ac.eps, d.paper_eps);
          x[k2[c]] = s_x[u][c];
          d.am[k2[c]] = s_m[u][c];
          d.av[k2[c]] = s_v[u][c];
        }
      } else {
        d.g[k2[0]] = gv[u];
        d.g[k2[1]] = gth[u];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// stage 5: generator gradients (+ Adam), objective reduction, step counter
// ---------------------------------------------------------------------------------------------

// Objective reduction, level 2, run by the closing kernel: per instance, the slots of its
// device blocks and of its fold blocks in fixed order (read through L2: other blocks wrote them),
// plus the closed-form soft-ReLU floor of the contingency term.
template <typename Real, typename Dc>
__device__ void final_reduce(const Dev<Real, Dc> &d, const InstTab &tab) {
  for (int b = 0; b < tab.n_inst; ++b) {
    const Inst &I = tab.I[b];
    Dc a[N_TERMS];
#pragma unroll
    for (int k = 0; k < N_TERMS; ++k) a[k] = DcOps<Dc>::zero();
    const int ns = I.gen_nb + I.fold_nb;
    for (int j = threadIdx.x; j < ns; j += NTHR) {
      const long long slot = j < I.gen_nb ? d.n_obj12 + I.gen_slot0 + j
                                          : d.n_obj12 + d.n_gen_slots + I.fold_slot0 + (j - I.gen_nb);
#pragma unroll
      for (int k = 0; k < N_TERMS; ++k) a[k] = DcOps<Dc>::add(a[k], ldcg(d.objp + slot * N_TERMS + k));
    }
    if (ns <= 32) {  // one warp holds every slot: a shuffle tree, no block barrier (block-uniform branch)
      if (threadIdx.x >= 32) continue;
#pragma unroll
      for (int k = 0; k < N_TERMS; ++k)
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) a[k] = DcOps<Dc>::add(a[k], DcOps<Dc>::shfl_down(a[k], q));
    } else {
      block_sum_terms(a);
    }
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int k = 0; k < N_TERMS; ++k) {
        double tv = to_double(a[k]);
        if (k == T_ZCTG) {
          double eps = d.eps64, beta = d.beta64;
          if (d.sched) {
            const long long it = sched_index(d);
            eps = d.sched[3 * it + 1];
            beta = d.sched[3 * it + 2];
          }
          tv += tab.I[b].hours * d.c_s64 * beta * eps * tab.I[b].nfloor_ctg;
        }
        d.terms[b * N_TERMS + k] = tv;
        tot += tv;
      }
      d.obj[b] = tot;
      if (d.trace) {
        const long long it = *d.step + d.step_off - *d.trace_step0;
        if (it >= 0 && it < d.trace_len) d.trace[it * tab.n_inst + b] = tot;
      }
    }
  }
}

// Device-level data of one (device, period), loaded before the wait (no stage writes it).
template <typename Real>
struct GenIn {
  int bus, zn, gb, b0, b1;  // bus, zone, generator-bus index, bid blocks [b0, b1)
  Real a, bl, cr, pmax, sg, p, q, r, u;
  double pmax64, ramp64;  // limits of the headroom and ramp residuals (formed in FP64)
  long long kp, kq, kr, ku;
  Real am[4], av[4], lo[4], hi[4];  // Adam moments and box of p, q, r, u (fused Adam only)
};

template <typename Real, typename Dc, bool ADAM>
__device__ GenIn<Real> gen_load(const Dev<Real, Dc> &d, const Inst &I, int t, int gl, const Real *x) {
  GenIn<Real> g;
  const int gg = I.gen0 + gl;
  g.bus = d.gen_bus[gg];
  g.zn = d.gen_zone[gg];
  g.gb = d.gen_gb[gg];
  g.b0 = d.blk_ptr[gg];
  g.b1 = d.blk_ptr[gg + 1];
  g.a = d.gen_a[gg];
  g.bl = d.gen_b[gg];
  g.cr = d.gen_cr[gg];
  g.pmax = d.gen_pmax[gg];
  g.pmax64 = d.lim_pmax[gg];
  g.ramp64 = d.lim_ramp[gg];
  g.sg = d.gen_sgn[gg];
  g.kp = I.x0 + 2LL * I.T * I.n + (long long)t * I.G + gl;
  g.kq = g.kp + (long long)I.T * I.G;
  g.kr = g.kq + (long long)I.T * I.G;
  g.ku = I.uc ? I.xu0 + (long long)t * I.G + gl : g.kp;
  g.p = x[g.kp];
  g.q = x[g.kq];
  g.r = x[g.kr];
  g.u = I.uc ? x[g.ku] : Real(1);
  if (ADAM) {
    const long long k4[4] = {g.kp, g.kq, g.kr, g.ku};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      g.am[c] = d.am[k4[c]];
      g.av[c] = d.av[k4[c]];
      g.lo[c] = d.lo[k4[c]];
      g.hi[c] = d.hi[k4[c]];
    }
  }
  return g;
}

// Energy cost (producer) or value (consumer) per hour of dispatch p and its derivative: bid blocks
// (Example 3) sum_l c_l max(min(p - P_{l-1}, w_l), 0), the derivative being the price of the block
// that p is entering (0 <= p - P_{l-1} < w_l); without blocks a p^2 + b p.
template <typename Real, typename Dc>
__device__ __forceinline__ void energy_cost(const Dev<Real, Dc> &d, const GenIn<Real> &g, Real &en, Real &den) {
  const Real p = g.p;
  if (g.b1 > g.b0) {
    en = 0;
    den = 0;
    for (int l = g.b0; l < g.b1; ++l) {
      const Real c = d.blk_c[l], w = d.blk_w[l], e = p - d.blk_lo[l];
      en += c * fmax(fmin(e, w), Real(0));
      if (e >= Real(0) && e < w) den += c;
    }
  } else {
    en = g.a * p * p + g.bl * p;
    den = 2 * g.a * p + g.bl;
  }
}

// Device terms of period t (energy cost or value, reserve cost, headroom, ramps; with on-status
// the on / startup / shutdown costs and the u-scaled limits; Eq. nlp_updated, Examples 2-4) and
// the gradient wrt p, q, r (, u), with the injection adjoint eta_gb - mean(eta) (Eqs. 2nd_lin_sys,
// correction) at the device's bus, signed by its role (producer +, consumer -);
// [+ the projected Adam update of p, q, r (, u)].
template <typename Real, typename Dc, bool ADAM>
__device__ void gen_update(const Dev<Real, Dc> &d, const Inst &I, int t, int gl, const GenIn<Real> &g, Dc eta,
                           const AdamCoef<Real> &ac, Obj3<Dc> &acc, Real *__restrict__ x) {
  const Real dt = d.dt[I.tp0 + t];
  const long long G = I.G;
  const Real p = g.p, q = g.q, r = g.r, u = g.u, sg = g.sg;
  const long long tb = I.tb0 + (long long)t * I.n;
  Real en, den;
  energy_cost(d, g, en, den);
  Real gp = dt * sg * den + sg * (DcOps<Dc>::to_real(eta) - d.dP[tb + g.bus]);
  Real gq = -sg * d.dQ[tb + g.bus];
  Real gr = dt * g.cr - d.dZ[I.tz0 + (long long)t * I.Z + g.zn];
  Real gu = 0;
  Real cost = dt * (sg * en + g.cr * r);
  const HP<Real> hp = hparams(d);
  const Real wr = d.rho * hp.beta;
  Real val, der;
  // residuals of the penalized linear constraints in FP64 (p, q, r, u are exact in it)
  const double p64 = p, q64 = q, r64 = r, u64 = u;
  soft_relu(Real(p64 + r64 - g.pmax64 * u64), hp.eps, val, der);  // u = 1 without on-status variables
  Real zh = wr * val;
  gp += wr * der;
  gr += wr * der;
  const long long ko = I.tg0 + (long long)t * G + gl;
  if (I.uc) {
    const int gg = I.gen0 + gl;
    gu -= g.pmax * (wr * der);
    const Real pmin = d.gen_pmin[gg], qmin = d.gen_qmin[gg], qmax = d.gen_qmax[gg];
    const double pmin64 = d.lim_pmin[gg], qmin64 = d.lim_qmin[gg], qmax64 = d.lim_qmax[gg];
    soft_relu(Real(pmin64 * u64 - p64), hp.eps, val, der);
    zh += wr * val;
    gp -= wr * der;
    gu += pmin * (wr * der);
    soft_relu(Real(q64 - qmax64 * u64), hp.eps, val, der);
    zh += wr * val;
    gq += wr * der;
    gu -= qmax * (wr * der);
    soft_relu(Real(qmin64 * u64 - q64), hp.eps, val, der);
    zh += wr * val;
    gq -= wr * der;
    gu += qmin * (wr * der);
    // on cost, startup max(u_t - u_{t-1}, 0) and shutdown max(u_{t-1} - u_t, 0) (Example 2)
    const Real csu = d.gen_csu[gg], csd = d.gen_csd[gg], con = d.gen_con[gg];
    const Real up = t >= 1 ? (ADAM ? d.uold[ko - G] : x[g.ku - G]) : d.gen_uinit[gg];
    const Real du = u - up;
    cost += dt * con * u + csu * fmax(du, Real(0)) + csd * fmax(-du, Real(0));
    gu += dt * con + (du > Real(0) ? csu : Real(0)) - (du < Real(0) ? csd : Real(0));
    if (t + 1 < I.T) {
      const Real dn = (ADAM ? d.uold[ko + G] : x[g.ku + G]) - u;
      gu -= (dn > Real(0) ? csu : Real(0)) - (dn < Real(0) ? csd : Real(0));
    }
  }
  acc.v[0] = DcOps<Dc>::from_real(cost);
  acc.v[1] = DcOps<Dc>::from_real(zh);
  if (t >= 1) {  // ramp terms of period t
    const double pp = ADAM ? d.pold[ko - G] : x[g.kp - G];
    const double lim = g.ramp64 * d.lim_dt[I.tp0 + t];
    Real v1, d1, v2, d2;
    soft_relu(Real(p64 - pp - lim), hp.eps, v1, d1);
    soft_relu(Real(pp - p64 - lim), hp.eps, v2, d2);
    acc.v[2] = DcOps<Dc>::from_real(wr * (v1 + v2));
    gp += wr * (d1 - d2);
  }
  if (t + 1 < I.T) {  // ramp terms of period t + 1 that involve p_t
    const double pn = ADAM ? d.pold[ko + G] : x[g.kp + G];
    const double lim = g.ramp64 * d.lim_dt[I.tp0 + t + 1];
    Real v1, d1, v2, d2;
    soft_relu(Real(pn - p64 - lim), hp.eps, v1, d1);
    soft_relu(Real(p64 - pn - lim), hp.eps, v2, d2);
    gp += wr * (d2 - d1);
  }
  if (ADAM) {
    const long long k4[4] = {g.kp, g.kq, g.kr, g.ku};
    const Real g4[4] = {gp, gq, gr, gu};
    const Real x4[4] = {p, q, r, u};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c == 3 && !I.uc) break;
      Real xk = x4[c], mk = g.am[c], vk = g.av[c];
      adam_update(xk, g4[c], mk, vk, g.lo[c], g.hi[c], ac.b1, ac.b2, ac.c1, ac.c2, ac.lr, ac.eps, d.paper_eps);
      x[k4[c]] = xk;
      d.am[k4[c]] = mk;
      d.av[k4[c]] = vk;
    }
  } else {
    d.g[g.kp] = gp;
    d.g[g.kq] = gq;
    d.g[g.kr] = gr;
    if (I.uc) d.g[g.ku] = gu;
  }
}

// The FP64 path's device update without on-status variables, one (period, device) pair over four
// lanes (part = lane & 3): 0 the energy cost, eta, the balance adjoint, the headroom and the ramp
// into period t, and p's update; 1 q's; 2 r's (with the headroom derivative from lane 0); 3 the
// ramp terms of period t + 1 that involve p_t (handed to lane 0).  Each gradient is summed in the
// order of gen_update, so the results are bitwise its; the dependent FP64 chain (square roots and
// divisions of the soft-ReLUs and of Adam) is about a third as long, and the work spreads over
// four times as many warps.  Every lane of the warp calls it (the shuffles are warp-wide).
template <typename Real, typename Dc, bool ADAM>
__device__ void gen_update_lanes(const Dev<Real, Dc> &d, const Inst &I, int t, int gl, int part, bool on,
                                 const GenIn<Real> &g, Dc eta, const AdamCoef<Real> &ac, Obj3<Dc> &acc,
                                 Real *__restrict__ x) {
  const long long G = I.G;
  const HP<Real> hp = hparams(d);
  const Real wr = d.rho * hp.beta;
  Real grad = 0, hd = 0, rp = 0;
  if (on) {
    const Real dt = d.dt[I.tp0 + t];
    const long long tb = I.tb0 + (long long)t * I.n;
    const long long ko = I.tg0 + (long long)t * G + gl;
    const double p64 = g.p;
    if (part == 0) {
      Real en, den, val, der;
      energy_cost(d, g, en, den);
      grad = dt * g.sg * den + g.sg * (DcOps<Dc>::to_real(eta) - d.dP[tb + g.bus]);
      acc.v[0] = DcOps<Dc>::from_real(dt * (g.sg * en + g.cr * g.r));
      soft_relu(Real(p64 + (double)g.r - g.pmax64), hp.eps, val, der);
      acc.v[1] = DcOps<Dc>::from_real(wr * val);
      hd = wr * der;
      grad += hd;
      if (t >= 1) {  // ramp terms of period t
        const double pp = ADAM ? d.pold[ko - G] : x[g.kp - G];
        const double lim = g.ramp64 * d.lim_dt[I.tp0 + t];
        Real v1, d1, v2, d2;
        soft_relu(Real(p64 - pp - lim), hp.eps, v1, d1);
        soft_relu(Real(pp - p64 - lim), hp.eps, v2, d2);
        acc.v[2] = DcOps<Dc>::from_real(wr * (v1 + v2));
        grad += wr * (d1 - d2);
      }
    } else if (part == 1) {
      grad = -g.sg * d.dQ[tb + g.bus];
    } else if (part == 2) {
      grad = dt * g.cr - d.dZ[I.tz0 + (long long)t * I.Z + g.zn];
    } else if (t + 1 < I.T) {  // ramp terms of period t + 1 that involve p_t
      const double pn = ADAM ? d.pold[ko + G] : x[g.kp + G];
      const double lim = g.ramp64 * d.lim_dt[I.tp0 + t + 1];
      Real v1, d1, v2, d2;
      soft_relu(Real(pn - p64 - lim), hp.eps, v1, d1);
      soft_relu(Real(p64 - pn - lim), hp.eps, v2, d2);
      rp = wr * (d2 - d1);
    }
  }
  const Real from3 = __shfl_xor_sync(0xffffffffu, rp, 3);  // lane 3 -> lane 0 of the pair
  const Real from0 = __shfl_xor_sync(0xffffffffu, hd, 2);  // lane 0 -> lane 2 of the pair
  if (!on || part == 3) return;
  if (part == 0 && t + 1 < I.T) grad += from3;
  if (part == 2) grad += from0;
  const long long k = part == 0 ? g.kp : part == 1 ? g.kq : g.kr;
  if (ADAM) {
    Real xk = part == 0 ? g.p : part == 1 ? g.q : g.r;
    Real mk = g.am[0], vk = g.av[0], lo = g.lo[0], hi = g.hi[0];
    if (part == 1) { mk = g.am[1]; vk = g.av[1]; lo = g.lo[1]; hi = g.hi[1]; }
    if (part == 2) { mk = g.am[2]; vk = g.av[2]; lo = g.lo[2]; hi = g.hi[2]; }
    adam_update(xk, grad, mk, vk, lo, hi, ac.b1, ac.b2, ac.c1, ac.c2, ac.lr, ac.eps, d.paper_eps);
    x[k] = xk;
    d.am[k] = mk;
    d.av[k] = vk;
  } else {
    d.g[k] = grad;
  }
}

// Transformer x of period t: dPhi/dtau from the AC terms (stage 3), and dPhi/dphi = -(the AC
// adjoint of delta) + b_sr dPhi/db, where dPhi/db = dz/dp_x - (E_hat eta)_x is the contingency
// term's phase-shift gradient (Eq. 2nd_lin_sys_phase plus the direct term of p = f + b);
// [+ the projected Adam update of tau and phi].
// Gradients of transformer xi in period t (tau: the AC terms; phi: the AC terms and the phase-shift
// flow b = b_sr phi, whose adjoint is dz/df of the branch plus the adjoint DC term `eterm`)
// [+ the projected Adam update].
template <typename Real, typename Dc, bool ADAM>
__device__ void xf_update(const Dev<Real, Dc> &d, const Inst &I, int t, int xi, Real eterm, Real *__restrict__ x,
                          const AdamCoef<Real> &ac) {
  const int j = d.xf_br[I.xf0 + xi];
  const long long e = I.tm0 + (long long)t * I.M + j;
  const Real gb = d.gF[e] + eterm;
  const Real gphi = -d.ad[e] + d.br_b[I.br0 + j] * gb;
  const Real gtau = d.atx[I.tx0 + (long long)t * I.X + xi];
  const long long kt = I.xtau0 + (long long)t * I.X + xi, kp = kt + (long long)I.T * I.X;
  if (ADAM) {
    adam_update(x[kt], gtau, d.am[kt], d.av[kt], d.lo[kt], d.hi[kt], ac.b1, ac.b2, ac.c1, ac.c2, ac.lr, ac.eps,
                d.paper_eps);
    adam_update(x[kp], gphi, d.am[kp], d.av[kp], d.lo[kp], d.hi[kp], ac.b1, ac.b2, ac.c1, ac.c2, ac.lr, ac.eps,
                d.paper_eps);
  } else {
    d.g[kt] = gtau;
    d.g[kp] = gphi;
  }
}

template <typename Real, typename Dc, bool ADAM>
__device__ void s5_xf(const Dev<Real, Dc> &d, const Inst &I, int t, int sub, Real *__restrict__ x,
                      const AdamCoef<Real> &ac) {
  const int xi = sub * NTHR + threadIdx.x;
  if (xi >= I.X) return;
  Real eterm;
  if (d.sp) {  // the adjoint term of the phase-shift flow is -(eta_f - eta_o) at the branch's ends
    const int j = d.xf_br[I.xf0 + xi];
    const int2 ft = d.br_end[I.br0 + j];
    const int pf = d.bus_pos[ft.x], po = d.bus_pos[ft.y];
    const Dc ef = pf >= 0 ? d.sp_th[(long long)pf * I.T + t] : DcOps<Dc>::zero();
    const Dc eo = po >= 0 ? d.sp_th[(long long)po * I.T + t] : DcOps<Dc>::zero();
    eterm = -DcOps<Dc>::to_real(DcOps<Dc>::add(ef, DcOps<Dc>::neg(eo)));
  } else {  // stage 4's product of the transformer's column
    eterm = DcOps<Dc>::to_real(d.gip[I.gi0 + (long long)t * (I.Gc + 1) + I.Gb + xi]);
  }
  xf_update<Real, Dc, ADAM>(d, I, t, xi, eterm, x, ac);
}

// Stage 5 (sparse DC mode, and the FP64 path's dense mode): devices of one period, with eta from the
// adjoint solve or from stage 4's products (whose columns already subtract the mean) | transformers
// of one period; the last block reduces the objective.
template <typename Real, typename Dc, bool ADAM>
__global__ void __launch_bounds__(NTHR) k_s5(const __grid_constant__ Dev<Real, Dc> d,
                                             const __grid_constant__ InstTab tab, const __grid_constant__ Spans S,
                                             Real *__restrict__ x) {
  const Where w = locate(S);
  const Inst &I = tab.I[tab.n_inst == 1 ? 0 : w.inst];  // one instance: no wait on the span search
  const int t = w.t;
  AdamCoef<Real> ac{};
  if (ADAM) ac = adam_coef(d);
  if (w.role == R_XF) {
    pdl_wait();
    s5_xf<Real, Dc, ADAM>(d, I, t, w.sub, x, ac);
  } else if (sizeof(Real) == 8 && !I.uc) {  // FP64 without on-status: four lanes per pair
    Obj3<Dc> acc = obj3<Dc>(T_COST, T_ZHEAD, T_ZRAMP);
    const int e = w.sub * I.gen_pb + (int)(threadIdx.x >> 2), part = threadIdx.x & 3;
    const bool on = (int)threadIdx.x < 4 * I.gen_pb && e < I.T * I.G;
    const int tg = on ? e / I.G : 0, gl = on ? e - tg * I.G : 0;
    const GenIn<Real> g = gen_load<Real, Dc, ADAM>(d, I, tg, gl, x);
    pdl_wait();
    Dc eta = DcOps<Dc>::zero();
    if (on && part == 0) {
      const Dc *et = d.gip + I.gi0 + (long long)tg * (I.Gc + 1);  // written by stage 4 or the adjoint solve
      eta = d.sp ? DcOps<Dc>::add(et[g.gb], DcOps<Dc>::neg(DcOps<Dc>::mul(et[I.Gc], DcOps<Dc>::inv_n(I)))) : et[g.gb];
    }
    if (threadIdx.x < 32) gen_update_lanes<Real, Dc, ADAM>(d, I, tg, gl, part, on, g, eta, ac, acc, x);
    write_obj(d.objp, d.n_obj12 + I.gen_slot0 + (blockIdx.x - I.gen_first), acc);
  } else {
    Obj3<Dc> acc = obj3<Dc>(T_COST, T_ZHEAD, T_ZRAMP);
    // (period, device) pairs packed densely over the instance's device blocks
    const int e = w.sub * I.gen_pb + threadIdx.x;
    const bool on = (int)threadIdx.x < I.gen_pb && e < I.T * I.G;
    const int tg = on ? e / I.G : 0, gl = on ? e - tg * I.G : 0;
    const GenIn<Real> g = gen_load<Real, Dc, ADAM>(d, I, tg, gl, x);
    pdl_wait();
    if (on) {
      const Dc *et = d.gip + I.gi0 + (long long)tg * (I.Gc + 1);  // written by stage 4 or the adjoint solve
      const Dc eta = d.sp ? DcOps<Dc>::add(et[g.gb], DcOps<Dc>::neg(DcOps<Dc>::mul(et[I.Gc], DcOps<Dc>::inv_n(I))))
                          : et[g.gb];
      gen_update<Real, Dc, ADAM>(d, I, tg, gl, g, eta, ac, acc, x);
    }
    write_obj(d.objp, d.n_obj12 + I.gen_slot0 + (blockIdx.x - I.gen_first), acc);
  }
}

// Right-hand side of the adjoint solve in the sparse mode (Eq. 2nd_lin_sys): w = E_hat^T Y_x dz/df
// at 32 positions x 8 periods per block, w_i = sum over incident branches of +-y_j dz/df_j (+ at
// the from-end); plus per-chunk partial sums of z1 . w = 1^T eta (n times the mean of eta, Eq.
// correction), finished in fixed order by the adjoint gather.
template <typename Real, typename Dc>
__device__ void s4_sdca(const Dev<Real, Dc> &d, const Inst &I, int tc, int sub) {
  const int t = tc * DCF_TC + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int pos = sub * 32 + lane;
  const bool on = t < I.T && pos < d.nr;
  const int q0 = on ? d.inc_ptr[pos] : 0, q1 = on ? d.inc_ptr[pos + 1] : 0;
  const Dc z1 = on ? d.z1[pos] : DcOps<Dc>::zero();
  pdl_wait();
  Dc w = DcOps<Dc>::zero();
  if (on) {
    const Real *gf = d.gF + I.tm0 + (long long)t * I.M;
    for (int q = q0; q < q1; ++q) {
      const int c = d.inc_code[q], j = c >> 1;
      const Real g = (c & 1) ? -gf[j] : gf[j];
      DcOps<Dc>::mac(w, d.ydc[I.br0 + j], DcOps<Dc>::from_real(g));
    }
    d.sp_rhs[(long long)pos * I.T + t] = w;
  }
  Dc s = DcOps<Dc>::mul(z1, w);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = DcOps<Dc>::add(s, DcOps<Dc>::shfl_down(s, o));
  if (lane == 0 && t < I.T) d.sp_part[(long long)sub * I.T + t] = s;
}

// Adjoint DC products and device updates of the dense DC mode (the last stage).  Warp w of the
// block takes column c = sub * 8 + w of period t:
//   eta'[t, c] = sum_m dz/df[t,m] A[c, m],   A[gb, m] = PTDF[m, gb] - (PTDF 1)[m] / n  (c = gb < Gb:
//   the injection adjoint at generator bus gb minus its mean over all buses, Eqs. 2nd_lin_sys and
//   correction, the mean folded into the column at set-up) | A[Gb + x, m] = PSDF[m, x] (transformer x,
//   Eq. 2nd_lin_sys_phase),
// lanes striding over the branches, a fixed-order shuffle reduction, and the sum broadcast to the
// warp; then (mixed path) its lanes update the devices at the bus, one per lane, or lane 0 the
// transformer (plans whose tab.fuse is set: small ones on the mixed path).  Otherwise the products are
// stored for stage 5, which updates 32 (FP64 path) or 256 devices per block: the FP64 pipe takes
// about as long for a warp with one active lane as for a full one, and large plans would get one
// objective slot per stage-4 block.
template <typename Real, typename Dc, bool ADAM, bool FUSE>
__device__ void s4_gbus(const Dev<Real, Dc> &d, const Inst &I, int t, int sub, const AdamCoef<Real> &ac,
                        Obj3<Dc> &acc, Real *__restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int c = sub * (NTHR / 32) + (threadIdx.x >> 5);
  const bool col = c < I.Gc;
  // data no earlier stage writes: the bus's first 32 devices (more take further rounds after the wait)
  int q0 = 0, q1 = 0;
  if (FUSE && col && c < I.Gb) {
    q0 = d.gb_ptr[I.gb0 + c];
    q1 = d.gb_ptr[I.gb0 + c + 1];
  }
  const bool dev0 = q0 + lane < q1;
  const int gl0 = dev0 ? d.gb_gen[q0 + lane] - I.gen0 : 0;
  const GenIn<Real> g = gen_load<Real, Dc, ADAM>(d, I, t, gl0, x);
  const Dc *A = d.ptdfaT + I.pg0 + (long long)(col ? c : 0) * I.M;
  if (col)  // the column is static: start bringing its lines to L2 before the wait
    for (long long off = (long long)lane * 128; off < (long long)I.M * (long long)sizeof(Dc); off += 32 * 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(A) + off));
  pdl_wait();
  if (!col) return;  // whole warp
  const Real *gf = d.gF + I.tm0 + (long long)t * I.M;
  Dc a[4] = {DcOps<Dc>::zero(), DcOps<Dc>::zero(), DcOps<Dc>::zero(), DcOps<Dc>::zero()};
  for (int m0 = 0; m0 < I.M; m0 += 8 * 32) {  // 8 strides per batch: their loads are issued together
    Dc av[8];
    Real gv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int m = m0 + k * 32 + lane;
      av[k] = m < I.M ? A[m] : DcOps<Dc>::zero();
      gv[k] = m < I.M ? gf[m] : Real(0);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) DcOps<Dc>::mac(a[k & 3], av[k], DcOps<Dc>::from_real(gv[k]));
  }
  Dc eta = DcOps<Dc>::add(DcOps<Dc>::add(a[0], a[1]), DcOps<Dc>::add(a[2], a[3]));
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) eta = DcOps<Dc>::add(eta, DcOps<Dc>::shfl_down(eta, k));
  if (!FUSE) {
    if (lane == 0) d.gip[I.gi0 + (long long)t * (I.Gc + 1) + c] = eta;
    return;
  }
  eta = DcOps<Dc>::bcast(eta);
  if (c >= I.Gb) {
    if (lane == 0) xf_update<Real, Dc, ADAM>(d, I, t, c - I.Gb, DcOps<Dc>::to_real(eta), x, ac);
    return;
  }
  Obj3<Dc> one = obj3<Dc>(T_COST, T_ZHEAD, T_ZRAMP);
  if (dev0) {
    gen_update<Real, Dc, ADAM>(d, I, t, gl0, g, eta, ac, one, x);
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.v[k] = DcOps<Dc>::add(acc.v[k], one.v[k]);
  }
  for (int q = q0 + 32 + lane; q < q1; q += 32) {  // a bus with more than 32 devices
    const int gl = d.gb_gen[q] - I.gen0;
    const GenIn<Real> g2 = gen_load<Real, Dc, ADAM>(d, I, t, gl, x);
    one = obj3<Dc>(T_COST, T_ZHEAD, T_ZRAMP);
    gen_update<Real, Dc, ADAM>(d, I, t, gl, g2, eta, ac, one, x);
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.v[k] = DcOps<Dc>::add(acc.v[k], one.v[k]);
  }
}

// Stage 4: bus gather of the branch-end adjoints (-> g_v, g_theta) [+ Adam on v, theta]; in the
// dense DC mode also the adjoint DC products with the device and transformer updates (the last
// stage: its last block reduces the objective); in the sparse mode the right-hand side of the
// adjoint solve.
template <typename Real, typename Dc, bool ADAM, bool FUSE>
__global__ void __launch_bounds__(NTHR) k_s4(const __grid_constant__ Dev<Real, Dc> d,
                                             const __grid_constant__ InstTab tab, const __grid_constant__ Spans S,
                                             Real *__restrict__ x) {
  const Where w = locate(S);
  const Inst &I = tab.I[tab.n_inst == 1 ? 0 : w.inst];  // one instance: no wait on the span search
  AdamCoef<Real> ac{};
  if (ADAM) ac = adam_coef(d);
  if (w.role == R_BUS) {
    s4_bus<Real, Dc, ADAM>(d, I, w.t, w.sub, x, ac);
  } else if (w.role == R_SDCA) {
    s4_sdca(d, I, w.t, w.sub);
  } else {  // R_GBUS
    Obj3<Dc> acc = obj3<Dc>(T_COST, T_ZHEAD, T_ZRAMP);
    s4_gbus<Real, Dc, ADAM, FUSE>(d, I, w.t, w.sub, ac, acc, x);
    if (FUSE) write_obj(d.objp, d.n_obj12 + I.gen_slot0 + (blockIdx.x - I.gen_first), acc);
  }
}

// ---------------------------------------------------------------------------------------------
// stand-alone projected Adam (Alg. 3) for qg_adam_step
// ---------------------------------------------------------------------------------------------

template <typename Real>
__global__ void __launch_bounds__(NTHR) k_adam(Real *__restrict__ x, Real *__restrict__ m, Real *__restrict__ v,
                                               const Real *__restrict__ g, const Real *__restrict__ lo,
                                               const Real *__restrict__ hi, long long n, long long *step,
                                               unsigned int *ticket, double lr, double b1, double b2, double eps,
                                               int paper_eps) {
  __shared__ Real sc[2];
  if (threadIdx.x == 0) bias_corr(b1, b2, *step, sc[0], sc[1]);
  __syncthreads();
  const Real c1 = sc[0], c2 = sc[1];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    adam_update(x[k], g[k], m[k], v[k], lo[k], hi[k], (Real)b1, (Real)b2, c1, c2, (Real)lr, (Real)eps, paper_eps);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    *step += 1;
    *ticket = 0;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------------------------
// sparse DC mode: Yhat^-1 through the sparse factor with a dense tail (no PTDF).  The factor
// Yhat = L diag(D_S, S) L^T eliminates the low-degree nodes first; with M1 = L_SS^-1 and
// M2 = -L_TS L_SS^-1 held explicitly as gather lists, a solve is
//   z_S = M1 b_S, z_T = b_T + M2 b_S  ->  x_T = S^-1 z_T  ->  x_S = M1^T (D_S^-1 z_S) + M2^T x_T,
// for all periods at once (node-major arrays [position][T]).
// ---------------------------------------------------------------------------------------------

// Forward right-hand sides p_inj[pos][t] = (dispatch at the bus) - load (blocks [0, nb)), and the
// mean injection mu_t = (sum_g p_gt - total load_t) / n (one block per period after those).
template <typename Real, typename Dc>
__global__ void __launch_bounds__(NTHR) k_sp_inj(const __grid_constant__ Dev<Real, Dc> d,
                                                 const __grid_constant__ Inst I, const Real *__restrict__ x, int nb) {
  const Real *p = x + I.x0 + 2LL * I.T * I.n;
  if ((int)blockIdx.x < nb) {
    const long long e = (long long)blockIdx.x * NTHR + threadIdx.x;
    if (e >= (long long)d.nr * I.T) return;
    const int pos = (int)(e / I.T), t = (int)(e % I.T);
    const int bus = d.pos_bus[pos], gb = d.pos_gb[pos];
    Dc s = DcOps<Dc>::neg(d.load_dc[I.tb0 + (long long)t * I.n + bus]);
    if (gb >= 0) {
      const int q0 = d.gb_ptr[I.gb0 + gb], q1 = d.gb_ptr[I.gb0 + gb + 1];
      for (int q = q0; q < q1; ++q) {
        const int gq = d.gb_gen[q];
        s = DcOps<Dc>::add(s, DcOps<Dc>::from_real(d.gen_sgn[gq] * p[(long long)t * I.G + (gq - I.gen0)]));
      }
    }
    if (I.X > 0) {  // - E^T b: a phase-shift flow leaves its from end and enters its to end
      for (int q = d.inc_ptr[pos]; q < d.inc_ptr[pos + 1]; ++q) {
        const int c = d.inc_code[q], j = c >> 1, xi = d.br_xf[I.br0 + j];
        if (xi < 0) continue;
        const Real b = d.br_b[I.br0 + j] * x[I.xtau0 + (long long)(I.T + t) * I.X + xi];
        s = DcOps<Dc>::add(s, DcOps<Dc>::from_real((c & 1) ? b : -b));
      }
    }
    d.sp_rhs[e] = s;
  } else {
    const int t = blockIdx.x - nb;
    Dc s = DcOps<Dc>::zero();
    for (int g = threadIdx.x; g < I.G; g += NTHR)
      s = DcOps<Dc>::add(s, DcOps<Dc>::from_real(d.gen_sgn[I.gen0 + g] * p[(long long)t * I.G + g]));
    s = block_sum_dc(s);
    if (threadIdx.x == 0)
      d.sp_mu[t] = DcOps<Dc>::mul(DcOps<Dc>::add(s, DcOps<Dc>::neg(d.ltot[I.tp0 + t])), DcOps<Dc>::inv_n(I));
  }
}

// Forward gather z = [M1; M2] b, lanes over periods.  Eliminated rows (a few entries each, their
// list holding the unit diagonal; one warp per row) store u = z / D; tail rows (the long M2 rows;
// one block per row, its 8 warps taking contiguous parts of the list, summed in warp order) store
// z_T = b_T + M2 b_S.  In the adjoint pass extra blocks finish 1^T eta from the per-chunk partials
// of stage 4 (one warp per period).
template <typename Real, typename Dc, bool ADJ>
__global__ void __launch_bounds__(NTHR) k_sp_fwd(const __grid_constant__ Dev<Real, Dc> d,
                                                 const __grid_constant__ Inst I, int nrow_blocks) {
  __shared__ Dc s_part[NTHR / 32][64];
  const int T = I.T;
  if (ADJ && (int)blockIdx.x >= nrow_blocks) {  // 1^T eta: one warp per period, lanes over the chunks
    pdl_wait();
    const int t = (blockIdx.x - nrow_blocks) * (NTHR / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= T) return;
    Dc s = DcOps<Dc>::zero();
    for (int c = lane; c < d.n_pchunk; c += 32) s = DcOps<Dc>::add(s, d.sp_part[(long long)c * T + t]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = DcOps<Dc>::add(s, DcOps<Dc>::shfl_down(s, o));
    if (lane == 0) d.gip[I.gi0 + (long long)t * (I.Gc + 1) + I.Gc] = s;
    return;
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nsb = (d.nS + NTHR / 32 - 1) / (NTHR / 32);
  const bool tail = (int)blockIdx.x >= nsb;
  const int row = tail ? d.nS + (blockIdx.x - nsb) : blockIdx.x * (NTHR / 32) + wid;
  const bool on = tail || row < d.nS;
  int e0 = on ? d.fw_ptr[row] : 0, e1 = on ? d.fw_ptr[row + 1] : 0;
  if (tail) {
    const int per = (e1 - e0 + NTHR / 32 - 1) / (NTHR / 32);
    e0 = min(e1, e0 + wid * per);
    e1 = min(e1, e0 + per);
  }
  pdl_wait();
  if (!on) return;  // whole warp (eliminated rows only)
  for (int t0 = 0; t0 < T; t0 += 64) {
    const int ta = t0 + lane, tb = t0 + 32 + lane;
    Dc a0 = DcOps<Dc>::zero(), a1 = DcOps<Dc>::zero();
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
      const Dc v = d.fw_val[e];
      const Dc *b = d.sp_rhs + (long long)d.fw_col[e] * T;
      if (ta < T) DcOps<Dc>::mac(a0, v, b[ta]);
      if (tb < T) DcOps<Dc>::mac(a1, v, b[tb]);
    }
    if (!tail) {
      const Dc di = d.dinv[row];
      Dc *u = d.sp_u + (long long)row * T;
      if (ta < T) u[ta] = DcOps<Dc>::mul(a0, di);
      if (tb < T) u[tb] = DcOps<Dc>::mul(a1, di);
    } else {
      s_part[wid][lane] = a0;
      s_part[wid][32 + lane] = a1;
      __syncthreads();
      if (wid == 0) {
        Dc z0 = s_part[0][lane], z1 = s_part[0][32 + lane];
#pragma unroll
        for (int w = 1; w < NTHR / 32; ++w) {
          z0 = DcOps<Dc>::add(z0, s_part[w][lane]);
          z1 = DcOps<Dc>::add(z1, s_part[w][32 + lane]);
        }
        const Dc *b = d.sp_rhs + (long long)row * T;
        Dc *z = d.sp_zt + (long long)(row - d.nS) * T;
        if (ta < T) z[ta] = DcOps<Dc>::add(b[ta], z0);
        if (tb < T) z[tb] = DcOps<Dc>::add(b[tb], z1);
      }
      __syncthreads();
    }
  }
}

// Dense tail x_T = S^-1 z_T (a dense contraction, but in double-FP32 for the FP64-accurate DC
// solve, so on the FP32 pipes).  Block (row tile, column split): SP_RB rows x the split's share of
// the columns x all periods (up to SP_TMAX per pass); thread (row group, period lane) holds 4 rows
// x 4 periods of accumulators; S^-1 and z_T staged through shared memory SP_BK columns at a time.
// Each split writes its partial sums; the last split of a row tile to finish (ticket) adds them in
// split order and writes u (for the backward gather) and the solution (forward pass) or the
// generator-bus adjoints (adjoint pass).
template <typename Real, typename Dc, bool ADJ>
__global__ void __launch_bounds__(NTHR, 2) k_sp_tail(const __grid_constant__ Dev<Real, Dc> d,
                                                  const __grid_constant__ Inst I, int ks, int kchunk) {
  __shared__ Dc s_s[SP_RB][SP_BK + 1];
  __shared__ Dc s_z[SP_BK][SP_TMAX];
  __shared__ bool last;
  const int T = I.T, m = d.nT;
  const int rt = blockIdx.x / ks, kp = blockIdx.x % ks;
  const int a0 = rt * SP_RB;
  const int b_lo = min(m, kp * kchunk), b_hi = min(m, b_lo + kchunk);
  const int rg = threadIdx.x >> 4, tc = threadIdx.x & 15;
  pdl_wait();
  for (int t0 = 0; t0 < T; t0 += SP_TMAX) {
    const int tn = min(SP_TMAX, T - t0);
    Dc acc[4][SP_TMAX / 16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < SP_TMAX / 16; ++j) acc[i][j] = DcOps<Dc>::zero();
    for (int b0 = b_lo; b0 < b_hi; b0 += SP_BK) {
      const int bn = min(SP_BK, b_hi - b0);
      __syncthreads();
#pragma unroll
      for (int e = threadIdx.x; e < SP_RB * SP_BK; e += NTHR) {
        const int rr = e / SP_BK, cc = e % SP_BK, ar = a0 + rr;
        s_s[rr][cc] = (ar < m && cc < bn) ? d.sinv[(long long)ar * m + b0 + cc] : DcOps<Dc>::zero();
      }
#pragma unroll
      for (int e = threadIdx.x; e < SP_BK * SP_TMAX; e += NTHR) {
        const int rr = e / SP_TMAX, cc = e % SP_TMAX;
        s_z[rr][cc] = (rr < bn && cc < tn) ? d.sp_zt[(long long)(b0 + rr) * T + t0 + cc] : DcOps<Dc>::zero();
      }
      __syncthreads();
#pragma unroll 2
      for (int k = 0; k < SP_BK; ++k) {
        Dc sv[4], zv[SP_TMAX / 16];
#pragma unroll
        for (int i = 0; i < 4; ++i) sv[i] = s_s[rg * 4 + i][k];
#pragma unroll
        for (int j = 0; j < SP_TMAX / 16; ++j) zv[j] = s_z[k][tc + 16 * j];
#pragma unroll
        for (int j = 0; j < SP_TMAX / 16; ++j)
          if (tc + 16 * j < tn)
#pragma unroll
            for (int i = 0; i < 4; ++i) DcOps<Dc>::mac(acc[i][j], sv[i], zv[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = a0 + rg * 4 + i;
      if (a >= m) continue;
#pragma unroll
      for (int j = 0; j < SP_TMAX / 16; ++j)
        if (tc + 16 * j < tn) d.sp_tpart[((long long)kp * m + a) * T + t0 + tc + 16 * j] = acc[i][j];
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(d.sp_tick + rt, 1u) == (unsigned)(ks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = threadIdx.x; e < SP_RB * T; e += NTHR) {
    const int a = a0 + e / T, t = e % T;
    if (a >= m) continue;
    Dc v = DcOps<Dc>::zero();
    for (int q = 0; q < ks; ++q) v = DcOps<Dc>::add(v, d.sp_tpart[((long long)q * m + a) * T + t]);
    const int pos = d.nS + a;
    d.sp_u[(long long)pos * T + t] = v;
    d.sp_th[(long long)pos * T + t] = v;  // forward: the angles; adjoint: eta (transformer gradients)
    if (ADJ) {
      const int gb = d.pos_gb[pos];
      if (gb >= 0) d.gip[I.gi0 + (long long)t * (I.Gc + 1) + gb] = v;
    }
  }
  if (threadIdx.x == 0) d.sp_tick[rt] = 0u;
}

// Backward gather x_S = M1^T u_S + M2^T u_T (u_S = D_S^-1 z_S, u_T = x_T), one warp per eliminated
// position: every one on the forward pass (angles), the generator buses and transformer ends on
// the adjoint pass.
template <typename Real, typename Dc, bool ADJ>
__global__ void __launch_bounds__(NTHR) k_sp_back(const __grid_constant__ Dev<Real, Dc> d,
                                                  const __grid_constant__ Inst I) {
  const int T = I.T;
  const int w = blockIdx.x * (NTHR / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int nrows = ADJ ? d.n_adj_rows : d.nS;
  const bool on = w < nrows;
  const int q = on ? (ADJ ? d.adj_rows[w] : w) : 0;
  const int e0 = on ? d.bw_ptr[q] : 0, e1 = on ? d.bw_ptr[q + 1] : 0;
  const int gb = (on && ADJ) ? d.pos_gb[q] : -1;
  pdl_wait();
  if (!on) return;
  for (int t0 = 0; t0 < T; t0 += 64) {
    const int ta = t0 + lane, tb = t0 + 32 + lane;
    Dc a0 = DcOps<Dc>::zero(), a1 = DcOps<Dc>::zero();
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
      const Dc v = d.bw_val[e];
      const Dc *u = d.sp_u + (long long)d.bw_col[e] * T;
      if (ta < T) DcOps<Dc>::mac(a0, v, u[ta]);
      if (tb < T) DcOps<Dc>::mac(a1, v, u[tb]);
    }
    if (ADJ && gb >= 0) {
      Dc *g = d.gip + I.gi0 + gb;
      if (ta < T) g[(long long)ta * (I.Gc + 1)] = a0;
      if (tb < T) g[(long long)tb * (I.Gc + 1)] = a1;
    }
    Dc *th = d.sp_th + (long long)q * T;  // forward: the angles; adjoint: eta (transformer gradients)
    if (ta < T) th[ta] = a0;
    if (tb < T) th[tb] = a1;
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------

template <typename Real>
size_t ctg_smem_bytes(int TB, bool score, bool lazy) {
  constexpr bool F64 = sizeof(Real) == 8;
  constexpr int TCH = ctg_tch<Real>();
  const size_t nch = (TB + TCH - 1) / TCH;
  return sizeof(float) * ((size_t)TB * (2 * CT_BM + 2 * CT_BK) + nch * (CT_BM + 4) +
                          (lazy ? (size_t)CT_TBATCH * (4 + nch) * CT_BM : 0)) +
         sizeof(Real) * ((size_t)TB * CT_BK + 2 * CT_BM + (size_t)TCH * (2 * CT_BM + 8 * CT_BK) +
                         (F64 ? (size_t)TB * (CT_BM + CT_BK) : 0) +
                         (score ? (size_t)TCH * 8 * CT_BK + (size_t)TB * CT_BK : 0));
}

// Record a timing event on s; inside stream capture it becomes an external event node.
static inline void mark(cudaEvent_t *ev, int k, cudaStream_t s) {
  if (!ev) return;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
  else cudaEventRecord(ev[k], s);
}

// Launch with programmatic stream serialization: the kernel may begin while its predecessor
// drains (no early trigger, so as the predecessor's blocks exit); it waits (griddepcontrol.wait)
// before reading the predecessor's results.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, size_t smem, cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTHR);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Closing kernel of an evaluation, or of a graph of n fused iterations: one block sums the
// objective of the last one from the slots the stage kernels left, then step += n (n = 0 for a
// plain evaluation).
template <typename Real, typename Dc>
__global__ void __launch_bounds__(NTHR) k_finish(const __grid_constant__ Dev<Real, Dc> d,
                                                 const __grid_constant__ InstTab tab, int n) {
  const long long step = *d.step;  // no stage kernel writes it
  pdl_wait();
  final_reduce(d, tab);
  if (threadIdx.x == 0) *d.step = step + n;
}

template <typename Real, typename Dc>
cudaError_t launch_finish(const Dev<Real, Dc> &d, const Plan &P, int n, cudaStream_t s) {
  return launch_pdl(k_finish<Real, Dc>, 1, 0, s, d, P.tab, n);
}

template <typename Real, typename Dc>
cudaError_t launch_eval(const Dev<Real, Dc> &d, const Plan &P, const void *xv, bool adam, bool close,
                        cudaStream_t s, cudaEvent_t *ev) {
  Real *x = const_cast<Real *>(static_cast<const Real *>(xv));
  const int o2 = P.s1.n_blocks;
  // with timing events between the kernels, launch them plainly so each event brackets one kernel
  const bool pdl = ev == nullptr;
  cudaError_t e = cudaSuccess;
  auto go = [&](auto kern, int grid, size_t smem, auto... args) {
    if (e != cudaSuccess) return;
    if (pdl) e = launch_pdl(kern, grid, smem, s, args...);
    else {
      kern<<<grid, NTHR, smem, s>>>(args...);
      e = cudaGetLastError();
    }
  };
  mark(ev, 0, s);
  nvtxRangePushA("qg stage 1");  // one NVTX range per stage, closed at the next stage's launch
  if (P.sp) {
    // sparse mode: forward solve theta' = Yhat^-1 p_inj before the flows of stage 1
    const Inst &I = P.tab.I[0];
    k_sp_inj<Real, Dc><<<P.sp_inj_blocks + I.T, NTHR, 0, s>>>(d, I, (const Real *)x, P.sp_inj_blocks);
    e = cudaGetLastError();
    go(k_sp_fwd<Real, Dc, false>, P.sp_fw_blocks, 0, d, I, P.sp_fw_blocks);
    if (P.sp_tail_blocks > 0) go(k_sp_tail<Real, Dc, false>, P.sp_tail_blocks, 0, d, I, P.sp_tail_ks, P.sp_tail_kc);
    if (P.sp_bw_blocks > 0) go(k_sp_back<Real, Dc, false>, P.sp_bw_blocks, 0, d, I);
    go(k_s1<Real, Dc>, P.s1.n_blocks, 0, d, P.tab, P.s1, (const Real *)x, 0);
  } else {
    k_s1<Real, Dc><<<P.s1.n_blocks, NTHR, 0, s>>>(d, P.tab, P.s1, x, 0);
    e = cudaGetLastError();
  }
  mark(ev, 1, s);
  nvtxRangePop();
  nvtxRangePushA("qg stage 2 (contingencies)");
  if (P.s2.n_blocks > 0) {  // no contingencies: nothing for stage 2
    if (P.ctg_lazy) go(k_ctg_margin<Real, Dc>, 152 * 4, 0, d, P.tab);
    const size_t sm2 = ctg_smem_bytes<Real>(P.maxTB, d.score != 0, P.ctg_lazy != 0);
    if (P.ctg_lazy) go(k_s2<Real, Dc, 2>, P.s2.n_blocks, sm2, d, P.tab, P.s2, (const Real *)x, o2);
    else if (P.ctg_bound) go(k_s2<Real, Dc, 1>, P.s2.n_blocks, sm2, d, P.tab, P.s2, (const Real *)x, o2);
    else go(k_s2<Real, Dc, 0>, P.s2.n_blocks, sm2, d, P.tab, P.s2, (const Real *)x, o2);
  }
  mark(ev, 2, s);
  nvtxRangePop();
  nvtxRangePushA("qg stage 3");
  if (P.tab.s3q > 1) go(k_s3<Real, Dc, S3_SPLIT_MAX>, P.s3.n_blocks, 0, d, P.tab, P.s3, (const Real *)x);
  else go(k_s3<Real, Dc, 1>, P.s3.n_blocks, 0, d, P.tab, P.s3, (const Real *)x);
  mark(ev, 3, s);
  nvtxRangePop();
  nvtxRangePushA("qg stage 4");
  // stage 4 with the device updates (small plans on the mixed path) or without them (a separate
  // instantiation: the fused role's registers would cost the lean one its occupancy)
  if (P.tab.fuse) {
    if (adam) go(k_s4<Real, Dc, true, true>, P.s4.n_blocks, 0, d, P.tab, P.s4, x);
    else go(k_s4<Real, Dc, false, true>, P.s4.n_blocks, 0, d, P.tab, P.s4, x);
  } else {
    if (adam) go(k_s4<Real, Dc, true, false>, P.s4.n_blocks, 0, d, P.tab, P.s4, x);
    else go(k_s4<Real, Dc, false, false>, P.s4.n_blocks, 0, d, P.tab, P.s4, x);
  }
  if (P.sp) {
    // sparse mode: adjoint solve eta = Yhat^-1 w at the generator buses, and 1^T eta
    const Inst &I = P.tab.I[0];
    go(k_sp_fwd<Real, Dc, true>, P.sp_fw_blocks + (I.T + NTHR / 32 - 1) / (NTHR / 32), 0, d, I, P.sp_fw_blocks);
    if (P.sp_tail_blocks > 0) go(k_sp_tail<Real, Dc, true>, P.sp_tail_blocks, 0, d, I, P.sp_tail_ks, P.sp_tail_kc);
    if (P.sp_bwa_blocks > 0) go(k_sp_back<Real, Dc, true>, P.sp_bwa_blocks, 0, d, I);
  }
  mark(ev, 4, s);
  nvtxRangePop();
  nvtxRangePushA("qg stage 5 + closing kernel");
  if (P.s5.n_blocks > 0) {  // the mixed path's dense mode updates the devices in stage 4
    if (adam) go(k_s5<Real, Dc, true>, P.s5.n_blocks, 0, d, P.tab, P.s5, x);
    else go(k_s5<Real, Dc, false>, P.s5.n_blocks, 0, d, P.tab, P.s5, x);
  }
  if (close) go(k_finish<Real, Dc>, 1, 0, d, P.tab, adam ? 1 : 0);  // the objective, step += 1 with Adam
  nvtxRangePop();
  mark(ev, 5, s);
  return e;
}


// The contingency kernel's dynamic shared-memory limit is a process-wide function attribute: it is
// only ever raised, so that creating a handle with smaller blocks never breaks an existing one.
template <typename Real, typename Dc>
cudaError_t prepare_eval(int maxTB, bool score, bool lazy) {
  static std::mutex mu;
  static size_t cur = 0;  // the same limit for every instantiation
  const size_t sm = ctg_smem_bytes<Real>(maxTB, score, lazy);
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(mu);
  if (sm <= cur) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_s2<Real, Dc, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_s2<Real, Dc, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_s2<Real, Dc, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) cur = sm;
  return e;
}

// Row maxima for the bound test of the contingency screen: lmax[g][m] = max |L[m, k]| over the 16
// outage columns k of group g, read through the same decoding as the screen (NaN pads and each
// outage's own branch ignored), capped at FLT_MAX, and 0 on the pad rows of the last 64-row tile.
__global__ void k_lmax(const void *__restrict__ lodf, int dtype, float *__restrict__ lmax, int M, int Kp,
                       long long l0, int rows, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i / rows), m = (int)(i % rows);
    float mx = 0.f;
    if (m < M)
      for (int q = 0; q < 4; ++q) {
        const int k = g * 16 + q * 4;
        if (k >= Kp) break;
        float v[4];
        lodf_load4(lodf, l0 + (long long)m * Kp + k, dtype, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) mx = fmaxf(mx, fabsf(v[j]));
      }
    lmax[i] = fminf(mx, FLT_MAX);
  }
}

cudaError_t launch_lmax(const void *lodf, int dtype, float *lmax, const Inst &I, cudaStream_t s) {
  const int rows = I.n_mt * CT_BM;
  const long long n = (long long)I.n_kt * 4 * rows;
  if (n == 0) return cudaSuccess;
  const int nb = (int)std::max(1LL, std::min((n + NTHR - 1) / NTHR, 152LL * 16));
  k_lmax<<<nb, NTHR, 0, s>>>(lodf, dtype, lmax + I.lm0, I.M, I.Kp, I.l0, rows, n);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_adam(Real *x, Real *m, Real *v, const Real *g, const Real *lo, const Real *hi, long long n,
                        long long *step, unsigned int *ticket, double lr, double b1, double b2, double eps,
                        int paper_eps, cudaStream_t s) {
  long long nb = (n + NTHR - 1) / NTHR;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  k_adam<Real><<<(int)nb, NTHR, 0, s>>>(x, m, v, g, lo, hi, n, step, ticket, lr, b1, b2, eps, paper_eps);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// batch rounding (Alg. 1) with a per-pair projection stand-in
// ---------------------------------------------------------------------------------------------

// Squared distance ((dp^2 + dq^2) + dr^2) + du^2 in FP64 without contraction (the same order and
// rounding as a plain left-to-right sum of squares).
__device__ __forceinline__ double dist4(double dp, double dq, double dr, double du) {
  double s = __dmul_rn(dp, dp);
  s = __dadd_rn(s, __dmul_rn(dq, dq));
  s = __dadd_rn(s, __dmul_rn(dr, dr));
  return __dadd_rn(s, __dmul_rn(du, du));
}

// Every (period, device) pair of one instance with on-status variables: the projection of (p, q, r, u)
// onto u in {0, 1} and the limits u implies (u = 1: pmin <= p <= pmax, 0 <= r <= rcap, p + r <= pmax,
// qmin <= q <= qmax, rcap = pmax for producers and 0 for consumers; u = 0: p = q = r = 0), whichever is
// nearer (ties to u = 1), and the squared distance moved (+inf for pairs already fixed).  The (p, r)
// projection is the box projection when it meets p + r <= pmax, else the nearest point of the segment
// p + r = pmax inside the box.  proj holds [u | p | q | r], each [T G].
template <typename Real, typename Dc>
__global__ void k_round_project(const __grid_constant__ Dev<Real, Dc> d, const __grid_constant__ Inst I,
                                const Real *__restrict__ x, const unsigned char *__restrict__ fixed,
                                double *__restrict__ dist, Real *__restrict__ proj) {
  const long long TG = (long long)I.T * I.G;
  const long long e = (long long)blockIdx.x * NTHR + threadIdx.x;
  if (e >= TG) return;
  const int g = (int)(e % I.G), gg = I.gen0 + g;
  const long long kp = I.x0 + 2LL * I.T * I.n + e, kq = kp + TG, kr = kq + TG, ku = I.xu0 + e;
  const double p0 = x[kp], q0 = x[kq], r0 = x[kr], u0 = x[ku];
  const double pmin = d.gen_pmin[gg], pmax = d.gen_pmax[gg], qmin = d.gen_qmin[gg], qmax = d.gen_qmax[gg];
  const double rcap = d.gen_sgn[gg] < 0 ? 0.0 : pmax;
  double p1 = fmin(fmax(p0, pmin), pmax), r1 = fmin(fmax(r0, 0.0), rcap);
  if (p1 + r1 > pmax) {
    double pl = 0.5 * (p0 + pmax - r0);
    pl = fmin(fmax(pl, fmax(pmin, pmax - rcap)), pmax);
    p1 = pl;
    r1 = pmax - pl;
  }
  const double q1 = fmin(fmax(q0, qmin), qmax);
  const double d1 = dist4(p0 - p1, q0 - q1, r0 - r1, u0 - 1.0);
  const double d0 = dist4(p0, q0, r0, u0);
  const bool on = d1 <= d0;
  const long long tg = I.tg0 + e;
  dist[tg] = fixed[tg] ? INFINITY : (on ? d1 : d0);
  const long long sTG = d.n_pairs;
  proj[tg] = on ? Real(1) : Real(0);
  proj[sTG + tg] = on ? (Real)p1 : Real(0);
  proj[2 * sTG + tg] = on ? (Real)q1 : Real(0);
  proj[3 * sTG + tg] = on ? (Real)r1 : Real(0);
}

// Fixes the listed pairs (indices into the instance's [T G] pairs) at their projection: x takes the
// projected p, q, r, u; the box pins u, and with u = 0 also p, q, r at 0, while with u = 1 it becomes
// the u = 1 limits (p in [pmin, pmax], q in [qmin, qmax], r in [0, rcap]).
template <typename Real, typename Dc>
__global__ void k_round_fix(const __grid_constant__ Dev<Real, Dc> d, const __grid_constant__ Inst I,
                            Real *__restrict__ x, Real *__restrict__ lo, Real *__restrict__ hi,
                            const int *__restrict__ idx, int n, unsigned char *__restrict__ fixed,
                            const Real *__restrict__ proj) {
  const int j = blockIdx.x * NTHR + threadIdx.x;
  if (j >= n) return;
  const long long TG = (long long)I.T * I.G, e = idx[j], tg = I.tg0 + e, sTG = d.n_pairs;
  const int gg = I.gen0 + (int)(e % I.G);
  const long long kp = I.x0 + 2LL * I.T * I.n + e, kq = kp + TG, kr = kq + TG, ku = I.xu0 + e;
  const Real u = proj[tg];
  x[ku] = u;
  x[kp] = proj[sTG + tg];
  x[kq] = proj[2 * sTG + tg];
  x[kr] = proj[3 * sTG + tg];
  lo[ku] = hi[ku] = u;
  if (u == Real(0)) {
    lo[kp] = hi[kp] = lo[kq] = hi[kq] = lo[kr] = hi[kr] = Real(0);
  } else {
    lo[kp] = d.gen_pmin[gg];
    hi[kp] = d.gen_pmax[gg];
    lo[kq] = d.gen_qmin[gg];
    hi[kq] = d.gen_qmax[gg];
    lo[kr] = Real(0);
    hi[kr] = d.gen_sgn[gg] < 0 ? Real(0) : d.gen_pmax[gg];
  }
  fixed[tg] = 1;
}

template <typename Real, typename Dc>
cudaError_t launch_round_project(const Dev<Real, Dc> &d, const Inst &I, const Real *x, const unsigned char *fixed,
                                 double *dist, Real *proj, cudaStream_t s) {
  const long long TG = (long long)I.T * I.G;
  if (TG == 0) return cudaSuccess;
  k_round_project<Real, Dc><<<(int)((TG + NTHR - 1) / NTHR), NTHR, 0, s>>>(d, I, x, fixed, dist, proj);
  return cudaGetLastError();
}

template <typename Real, typename Dc>
cudaError_t launch_round_fix(const Dev<Real, Dc> &d, const Inst &I, Real *x, Real *lo, Real *hi, const int *idx,
                             int n, unsigned char *fixed, const Real *proj, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_round_fix<Real, Dc><<<(n + NTHR - 1) / NTHR, NTHR, 0, s>>>(d, I, x, lo, hi, idx, n, fixed, proj);
  return cudaGetLastError();
}

template cudaError_t launch_round_project<double, double>(const Dev<double, double> &, const Inst &, const double *,
                                                          const unsigned char *, double *, double *, cudaStream_t);
template cudaError_t launch_round_project<float, df32>(const Dev<float, df32> &, const Inst &, const float *,
                                                       const unsigned char *, double *, float *, cudaStream_t);
template cudaError_t launch_round_fix<double, double>(const Dev<double, double> &, const Inst &, double *, double *,
                                                      double *, const int *, int, unsigned char *, const double *,
                                                      cudaStream_t);
template cudaError_t launch_round_fix<float, df32>(const Dev<float, df32> &, const Inst &, float *, float *, float *,
                                                   const int *, int, unsigned char *, const float *, cudaStream_t);

template cudaError_t launch_eval<double, double>(const Dev<double, double> &, const Plan &, const void *, bool,
                                                 bool, cudaStream_t, cudaEvent_t *);
template cudaError_t launch_eval<float, df32>(const Dev<float, df32> &, const Plan &, const void *, bool, bool,
                                              cudaStream_t, cudaEvent_t *);
template cudaError_t prepare_eval<double, double>(int, bool, bool);
template cudaError_t launch_finish<double, double>(const Dev<double, double> &, const Plan &, int, cudaStream_t);
template cudaError_t launch_finish<float, df32>(const Dev<float, df32> &, const Plan &, int, cudaStream_t);
template cudaError_t prepare_eval<float, df32>(int, bool, bool);
template cudaError_t launch_adam<double>(double *, double *, double *, const double *, const double *, const double *,
                                         long long, long long *, unsigned int *, double, double, double, double, int,
                                         cudaStream_t);
template cudaError_t launch_adam<float>(float *, float *, float *, const float *, const float *, const float *,
                                        long long, long long *, unsigned int *, double, double, double, double, int,
                                        cudaStream_t);

}  // namespace qg
