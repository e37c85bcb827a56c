// Device kernels of one QuasiGrad objective + gradient evaluation and of the
// projected Adam step, for GB300 (sm_103a).
//
// One evaluation is a fixed sequence of short kernels (captured into a CUDA
// graph by the host for the Adam loop):
//   k_fwd1   AC branch flows (pi model) + thermal penalty; zonal reserve sums
//   k_fwd2   bus P/Q balance by CSR gather + soft-abs penalty; DC injections
//   k_dc     base DC solve: theta = Yhat^-1 (p_inj - mean) as a dense apply
//   k_ctg    post-contingency flows F = f_m + L[m,k] f_k, overload penalty and
//            both backward sums (the rank-1 SMW correction of Eq. rank_correct
//            written in flow space)
//   k_adj1   adjoint right-hand side w = E^T Y_x dz/df (Eq. 2nd_lin_sys)
//   k_dc     adjoint DC solve and slack correction eta - mean(eta) (Eq. correction)
//   k_bwd1   branch-end adjoints (chain rule through the pi-model flows)
//   k_bwd2   bus gather of the branch-end adjoints; generator gradients
//   k_obj    deterministic FP64 reduction of the objective terms
// No floating-point atomics are used: every sum has a fixed order, so repeated
// evaluations are bitwise identical.
//
// Every block of the entity kernels reads a descriptor (instance, period,
// entity slice, role), so instances of different sizes share one launch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "qg_internal.h"

namespace qg {

// ---------------------------------------------------------------------------------------------
// double-FP32 arithmetic (Dekker / Knuth error-free transformations)
// ---------------------------------------------------------------------------------------------

// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float hi = __fadd_rn(s, e);
  float lo = __fsub_rn(e, __fsub_rn(hi, s));
  return {hi, lo};
}

// acc += a * b with a, b double-FP32: TwoProd via FMA for hi*hi, first-order cross terms.
__device__ __forceinline__ void df_mac(df32 &acc, df32 a, df32 b) {
  float p = __fmul_rn(a.hi, b.hi);
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
  __device__ static double sub(double a, double b) { return a - b; }
  __device__ static void mac(double &acc, double a, double b) { acc = fma(a, b, acc); }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double inv_n(const Inst &I) { return I.inv_n; }
  __device__ static double to_real(double a) { return a; }
  __device__ static double shfl_down(double a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
};

template <>
struct DcOps<df32> {
  __device__ static df32 zero() { return {0.f, 0.f}; }
  __device__ static df32 from_real(float v) { return {v, 0.f}; }
  __device__ static df32 add(df32 a, df32 b) { return df_add(a, b); }
  __device__ static df32 sub(df32 a, df32 b) { return df_add(a, {-b.hi, -b.lo}); }
  __device__ static void mac(df32 &acc, df32 a, df32 b) { df_mac(acc, a, b); }
  __device__ static df32 mul(df32 a, df32 b) {
    df32 r = {0.f, 0.f};
    df_mac(r, a, b);
    return r;
  }
  __device__ static df32 inv_n(const Inst &I) { return {I.inv_n_hi, I.inv_n_lo}; }
  __device__ static float to_real(df32 a) { return __fadd_rn(a.hi, a.lo); }
  __device__ static df32 shfl_down(df32 a, int o) {
    return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
  }
};

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ double dsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float dsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ void dsincos(double a, double *s, double *c) { sincos(a, s, c); }
__device__ __forceinline__ void dsincos(float a, float *s, float *c) { sincosf(a, s, c); }

// soft-ReLU sigma_s(u) = sqrt(max(u,0)^2 + eps^2) and its derivative (Sec. II-C footnote)
template <typename Real>
__device__ __forceinline__ void soft_relu(Real u, Real eps, Real &val, Real &der) {
  Real m = u > Real(0) ? u : Real(0);
  Real s = dsqrt(m * m + eps * eps);
  val = s;
  der = s > Real(0) ? m / s : Real(0);
}

// soft-abs |u|_s = sqrt(u^2 + eps^2) and its derivative
template <typename Real>
__device__ __forceinline__ void soft_abs(Real u, Real eps, Real &val, Real &der) {
  Real s = dsqrt(u * u + eps * eps);
  val = s;
  der = s > Real(0) ? u / s : Real(0);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of NV doubles; result valid in thread 0.  blockDim.x <= 1024.
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
  __shared__ double red[32][NV];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[wid][k] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? red[lane][k] : 0.0;
      v[k] = warp_sum(s);
    }
  }
  __syncthreads();
}

// Deterministic block sum of one Dc value; result valid in thread 0.
template <typename Dc>
__device__ Dc block_sum_dc(Dc v) {
  __shared__ Dc red[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = DcOps<Dc>::add(v, DcOps<Dc>::shfl_down(v, o));
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    Dc s = lane < nw ? red[lane] : DcOps<Dc>::zero();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = DcOps<Dc>::add(s, DcOps<Dc>::shfl_down(s, o));
    v = s;
  }
  __syncthreads();
  return v;
}

__device__ __forceinline__ void write_terms(double *objp, int slot, const double (&t)[N_TERMS]) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N_TERMS; ++k) objp[(long long)slot * N_TERMS + k] = t[k];
  }
}

template <typename Real>
__device__ __forceinline__ Real real_nan();
template <>
__device__ __forceinline__ double real_nan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <>
__device__ __forceinline__ float real_nan<float>() { return __int_as_float(0x7fc00000); }

// x block accessors (five period-major blocks per instance)
template <typename Real>
struct XView {
  const Real *v, *th, *p, *q, *r;
  __device__ XView(const Real *x, const Inst &I) {
    long long n = I.n, G = I.G, T = I.T;
    v = x + I.x0;
    th = v + T * n;
    p = th + T * n;
    q = p + T * G;
    r = q + T * G;
  }
};

// ---------------------------------------------------------------------------------------------
// k_fwd1: AC branch flows + thermal penalty (R_BRANCH); zonal reserve shortfall (R_ZONE)
// ---------------------------------------------------------------------------------------------

template <typename Real, typename Dc>
__global__ void __launch_bounds__(256) k_fwd1(Dev<Real, Dc> d, const Blk *__restrict__ blks, const Real *__restrict__ x,
                                              int slot0) {
  const Blk b = blks[blockIdx.x];
  const Inst I = d.inst[b.inst];
  const int t = b.t;
  const Real dt = d.dt[I.tp0 + t];
  double acc[N_TERMS] = {0, 0, 0, 0, 0, 0, 0, 0};
  XView<Real> X(x, I);
  if (b.role == R_BRANCH) {
    const int j = b.base + threadIdx.x;
    if (j < I.M) {
      const int jg = I.br0 + j;
      const int f = d.br_from[jg] - I.bus0, o = d.br_to[jg] - I.bus0;
      const Real vf = X.v[(long long)t * I.n + f], vo = X.v[(long long)t * I.n + o];
      const Real dl = X.th[(long long)t * I.n + f] - X.th[(long long)t * I.n + o];
      Real sn, cs;
      dsincos(dl, &sn, &cs);
      const Real g = d.br_g[jg], bb = d.br_b[jg], bc = d.br_bc[jg];
      const Real vv = vf * vo;
      // Pi model, written without the cancellation of g vf^2 against g vf vo cos(d):
      //   p_fr = g vf (vf - vo) + g vf vo (1 - cos d) - b vf vo sin d, and likewise for the others,
      // with 1 - cos d = sin^2 d / (1 + cos d) while cos d > 0.
      const Real dv = vf - vo;
      const Real omc = cs > Real(0) ? sn * sn / (Real(1) + cs) : Real(1) - cs;
      const Real hch = bc - bb;  // b_ch / 2
      const Real pf = g * vf * dv + g * vv * omc - bb * vv * sn;
      const Real pt = -g * vo * dv + g * vv * omc + bb * vv * sn;
      const Real qf = -bb * vf * dv - hch * vf * vf - bb * vv * omc - g * vv * sn;
      const Real qt = bb * vo * dv - hch * vo * vo - bb * vv * omc + g * vv * sn;
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
      const Real smax = d.br_smax[jg];
      Real val;
      if (sm2 > smax * smax) {
        Real u = dsqrt(sm2) - smax, der;
        soft_relu(u, d.eps, val, der);
      } else {
        val = d.eps;
      }
      acc[T_ZS] = (double)(dt * d.c_s * d.beta * val);
    }
  } else if (b.role == R_ZONE) {
    const int z = b.base + threadIdx.x;
    if (z < I.Z) {
      const int zg = I.zone0 + z;
      Real sr = 0;
      for (int e = d.zgen_ptr[zg]; e < d.zgen_ptr[zg + 1]; ++e) sr += X.r[(long long)t * I.G + (d.zgen[e] - I.gen0)];
      const Real u = d.rreq[I.tz0 + (long long)t * I.Z + z] - sr;
      Real val, der;
      soft_relu(u, d.eps, val, der);
      const Real w = dt * d.c_rz * d.beta;
      d.dZ[I.tz0 + (long long)t * I.Z + z] = w * der;
      acc[T_ZRZ] = (double)(w * val);
    }
  }
  block_sum(acc);
  write_terms(d.objp, slot0 + blockIdx.x, acc);
}

// ---------------------------------------------------------------------------------------------
// k_fwd2: bus balance (Example 4) by CSR gather; DC injections and their per-block sums
// ---------------------------------------------------------------------------------------------

template <typename Real, typename Dc>
__global__ void __launch_bounds__(256) k_fwd2(Dev<Real, Dc> d, const Blk *__restrict__ blks, const Real *__restrict__ x,
                                              int slot0) {
  const Blk b = blks[blockIdx.x];
  const Inst I = d.inst[b.inst];
  const int t = b.t;
  const Real dt = d.dt[I.tp0 + t];
  double acc[N_TERMS] = {0, 0, 0, 0, 0, 0, 0, 0};
  XView<Real> X(x, I);
  Dc inj = DcOps<Dc>::zero();
  const int i = b.base + threadIdx.x;
  if (i < I.n) {
    const int ig = I.bus0 + i;
    const long long ti = I.tb0 + (long long)t * I.n + i;
    const Real lp = d.load_p[ti], lq = d.load_q[ti];
    Real P = lp, Q = lq;
    const long long tm = I.tm0 + (long long)t * I.M - I.br0;
    for (int e = d.inc_ptr[ig]; e < d.inc_ptr[ig + 1]; ++e) {
      const int code = d.inc[e];
      const long long k = tm + (code >> 1);
      if (code & 1) {
        P += d.pt[k];
        Q += d.qt[k];
      } else {
        P += d.pf[k];
        Q += d.qf[k];
      }
    }
    inj = DcOps<Dc>::from_real(-lp);
    for (int e = d.bgen_ptr[ig]; e < d.bgen_ptr[ig + 1]; ++e) {
      const long long k = (long long)t * I.G + (d.bgen[e] - I.gen0);
      const Real pg = X.p[k];
      P -= pg;
      Q -= X.q[k];
      inj = DcOps<Dc>::add(inj, DcOps<Dc>::from_real(pg));
    }
    Real vp, dp, vq, dq;
    soft_abs(P, d.eps, vp, dp);
    soft_abs(Q, d.eps, vq, dq);
    const Real wp = dt * d.c_p * d.beta, wq = dt * d.c_q * d.beta;
    d.dP[ti] = wp * dp;
    d.dQ[ti] = wq * dq;
    d.pinj[ti] = inj;
    acc[T_ZP] = (double)(wp * vp);
    acc[T_ZQ] = (double)(wq * vq);
  }
  Dc s = block_sum_dc(inj);
  if (threadIdx.x == 0) d.mupart[I.ib0 + (long long)t * I.n_ib + b.ib] = s;
  block_sum(acc);
  write_terms(d.objp, slot0 + blockIdx.x, acc);
}

// ---------------------------------------------------------------------------------------------
// k_dc: dense apply of the reduced-Laplacian inverse (ref row/col zero), all periods at once.
//   FWD: out[t,i] = sum_j Z[i,j] pinj[t,j] - mean_t(pinj) * z1[i]        (base angles, Eq. Yb_solve)
//   ADJ: out[t,i] = sum_j Z[i,j] w[t,j]   - (1/n) sum_j z1[j] w[t,j]     (Eq. 2nd_lin_sys + Eq. correction)
// One warp per row i; lanes stride over j; TC periods per pass.
// ---------------------------------------------------------------------------------------------

constexpr int DC_ROWS = 4;  // warps (rows) per block
constexpr int DC_TC = 8;    // periods per pass

template <typename Real, typename Dc, bool ADJ>
__global__ void __launch_bounds__(DC_ROWS * 32) k_dc(Dev<Real, Dc> d, const DcTile *__restrict__ tiles) {
  const DcTile tile = tiles[blockIdx.x];
  const Inst I = d.inst[tile.inst];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = tile.i0 + wid;
  const Dc *in = ADJ ? d.w : d.pinj;
  const Dc *part = ADJ ? d.spart : d.mupart;
  Dc *out = ADJ ? d.ginj : d.th;
  if (i >= I.n) return;
  const Dc *zrow = d.zinv + I.z0 + (long long)i * I.n;
  const Dc zi1 = d.z1[I.bus0 + i];
  const Dc invn = DcOps<Dc>::inv_n(I);
  for (int t0 = 0; t0 < I.T; t0 += DC_TC) {
    Dc acc[DC_TC];
#pragma unroll
    for (int tt = 0; tt < DC_TC; ++tt) acc[tt] = DcOps<Dc>::zero();
    const int tn = min(DC_TC, I.T - t0);
    for (int j = lane; j < I.n; j += 32) {
      const Dc zij = zrow[j];
#pragma unroll
      for (int tt = 0; tt < DC_TC; ++tt) {
        if (tt < tn) DcOps<Dc>::mac(acc[tt], zij, in[I.tb0 + (long long)(t0 + tt) * I.n + j]);
      }
    }
#pragma unroll
    for (int tt = 0; tt < DC_TC; ++tt) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[tt] = DcOps<Dc>::add(acc[tt], DcOps<Dc>::shfl_down(acc[tt], o));
    }
    if (lane == 0) {
      for (int tt = 0; tt < tn; ++tt) {
        const int t = t0 + tt;
        Dc s = DcOps<Dc>::zero();
        for (int k = 0; k < I.n_ib; ++k) s = DcOps<Dc>::add(s, part[I.ib0 + (long long)t * I.n_ib + k]);
        Dc corr;
        if (ADJ) {
          corr = DcOps<Dc>::mul(s, invn);  // mean of eta (eta_ref = 0)
        } else {
          corr = DcOps<Dc>::mul(DcOps<Dc>::mul(s, invn), zi1);  // mean injection times Z 1
        }
        out[I.tb0 + (long long)t * I.n + i] = DcOps<Dc>::sub(acc[tt], corr);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// k_ctg: contingency overloads and their backward sums (A8).
// Tile of BM monitored branches x BK outages, looping over every period with the
// line-outage block held in registers.  For outage k and monitored branch m:
//   F = f_m + L[m,k] f_k,  s = sqrt(F^2 + qmax2_m),  z += w sigma_s(s - s_ctg_m)
// Violations are rare: the common path is two FMAs and a compare per element;
// the soft-ReLU floor (eps per non-violating element) is added in closed form by k_obj.
// Pad elements and the outaged branch itself carry L = NaN, so F is NaN and the
// compare is false (they are never monitored).
// ---------------------------------------------------------------------------------------------

constexpr int CT_BM = 64, CT_BK = 64, CT_RM = 8;  // 8 warps x 8 rows, 32 lanes x 2 columns

template <typename Real>
__device__ __forceinline__ Real load_lodf(const void *base, long long idx, int dtype);
template <>
__device__ __forceinline__ double load_lodf<double>(const void *base, long long idx, int) {
  return static_cast<const double *>(base)[idx];
}
template <>
__device__ __forceinline__ float load_lodf<float>(const void *base, long long idx, int dtype) {
  if (dtype == QG_LODF_BF16) {
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(base)[idx]);
  } else if (dtype == QG_LODF_BF16X2) {
    const __nv_bfloat162 h = static_cast<const __nv_bfloat162 *>(base)[idx];
    return __bfloat162float(h.x) + __bfloat162float(h.y);
  }
  return static_cast<const float *>(base)[idx];
}

template <typename Real, typename Dc>
__global__ void __launch_bounds__(256) k_ctg(Dev<Real, Dc> d, const CtgTile *__restrict__ tiles, int slot0,
                                             int lodf_dtype) {
  extern __shared__ unsigned char smem_raw[];
  const CtgTile tile = tiles[blockIdx.x];
  const Inst I = d.inst[tile.inst];
  const int T = I.T;
  Real *s_fm = reinterpret_cast<Real *>(smem_raw);  // [T][BM] base flow on monitored branch
  Real *s_qs = s_fm + T * CT_BM;                     // [T][BM] qmax2 - sctg^2
  Real *s_q2 = s_qs + T * CT_BM;                     // [T][BM] qmax2
  Real *s_fk = s_q2 + T * CT_BM;                     // [T][BK] base flow on the outaged branch
  Real *s_sc = s_fk + T * CT_BK;                     // [BM] sctg
  Real *s_gm = s_sc + CT_BM;                         // [BM]
  Real *s_gq = s_gm + CT_BM;                         // [BM]
  Real *s_gk = s_gq + CT_BM;                         // [8][BK]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  // --- stage base flows f = y (theta_f - theta_o) of every period for the tile's rows/columns
  for (int e = threadIdx.x; e < T * (CT_BM + CT_BK); e += blockDim.x) {
    const int t = e / (CT_BM + CT_BK), c = e % (CT_BM + CT_BK);
    int jg = -1;
    if (c < CT_BM) {
      const int m = tile.m0 + c;
      if (m < I.M) jg = I.br0 + m;
    } else {
      const int k = tile.k0 + (c - CT_BM);
      if (k < I.K) jg = d.ctg_br[I.ctg0 + k];
    }
    Real f = 0;
    if (jg >= 0) {
      const long long tb = I.tb0 + (long long)t * I.n - I.bus0;
      const Dc a = d.th[tb + d.br_from[jg]], bth = d.th[tb + d.br_to[jg]];
      f = d.br_y[jg] * DcOps<Dc>::to_real(DcOps<Dc>::sub(a, bth));
    }
    if (c < CT_BM) {
      s_fm[t * CT_BM + c] = f;
      Real q2 = 0, sc = Real(1e30);
      if (jg >= 0) {
        q2 = d.qm2[I.tm0 + (long long)t * I.M + (jg - I.br0)];
        sc = d.br_sctg[jg];
      }
      s_q2[t * CT_BM + c] = q2;
      s_qs[t * CT_BM + c] = q2 - sc * sc;
      if (t == 0) s_sc[c] = sc;
    } else {
      s_fk[t * CT_BK + (c - CT_BM)] = f;
    }
  }
  // --- this thread's block of the line-outage matrix
  Real Lr[CT_RM][2];
  int kk[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) kk[a] = tile.k0 + lane + 32 * a;
#pragma unroll
  for (int bq = 0; bq < CT_RM; ++bq) {
    const int m = tile.m0 + wid * CT_RM + bq;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int k = kk[a];
      Real v = real_nan<Real>();
      if (m < I.M && k < I.K && d.ctg_br[I.ctg0 + k] != I.br0 + m)
        v = load_lodf<Real>(d.lodf, I.l0 + (long long)m * I.K + k, lodf_dtype);
      Lr[bq][a] = v;
    }
  }
  __syncthreads();

  double obj = 0.0;
  const Real eps = d.eps;
  for (int t = 0; t < T; ++t) {
    const Real w = d.dt[I.tp0 + t] * d.c_s * d.beta;
    Real gm[CT_RM], gq[CT_RM], gk[2] = {0, 0};
    bool any = false;
#pragma unroll
    for (int bq = 0; bq < CT_RM; ++bq) {
      gm[bq] = 0;
      gq[bq] = 0;
      const int mm = wid * CT_RM + bq;
      const Real fm = s_fm[t * CT_BM + mm], qs = s_qs[t * CT_BM + mm];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const Real F = fm + Lr[bq][a] * s_fk[t * CT_BK + lane + 32 * a];
        const Real e = F * F + qs;
        if (e > Real(0)) {  // rare: a post-contingency overload
          any = true;
          const Real s = dsqrt(F * F + s_q2[t * CT_BM + mm]);
          const Real u = s - s_sc[mm];
          Real val, der;
          soft_relu(u, eps, val, der);
          obj += (double)(w * (val - eps));
          const Real dd = w * der / s;  // d z / d F = w sigma' F / s
          gm[bq] += dd * F;
          gk[a] += dd * F * Lr[bq][a];
          gq[bq] += Real(0.5) * dd;       // d z / d qmax2 = w sigma' / (2 s)
        }
      }
    }
    const bool block_any = __syncthreads_or(any);
    const long long pm_row = I.pm0 + ((long long)tile.kt * T + t) * I.M;
    const long long pk_row = I.pk0 + ((long long)tile.mt * T + t) * I.K;
    if (!block_any) {
      if (threadIdx.x < CT_BM) {
        const int m = tile.m0 + threadIdx.x;
        if (m < I.M) {
          d.pm[pm_row + m] = 0;
          d.pq[pm_row + m] = 0;
        }
      } else if (threadIdx.x < CT_BM + CT_BK) {
        const int k = tile.k0 + threadIdx.x - CT_BM;
        if (k < I.K) d.pk[pk_row + k] = 0;
      }
      continue;
    }
    // row sums over the tile's outages: lanes (and the two columns per lane)
#pragma unroll
    for (int bq = 0; bq < CT_RM; ++bq) {
      Real v1 = warp_sum(gm[bq]);
      Real v2 = warp_sum(gq[bq]);
      if (lane == 0) {
        s_gm[wid * CT_RM + bq] = v1;
        s_gq[wid * CT_RM + bq] = v2;
      }
    }
    // column sums over the tile's monitored rows: across the 8 warps, fixed order
    s_gk[wid * CT_BK + lane] = gk[0];
    s_gk[wid * CT_BK + lane + 32] = gk[1];
    __syncthreads();
    if (threadIdx.x < CT_BM) {
      const int m = tile.m0 + threadIdx.x;
      if (m < I.M) {
        d.pm[pm_row + m] = s_gm[threadIdx.x];
        d.pq[pm_row + m] = s_gq[threadIdx.x];
      }
    } else if (threadIdx.x < CT_BM + CT_BK) {
      const int c = threadIdx.x - CT_BM;
      const int k = tile.k0 + c;
      Real s = 0;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) s += s_gk[ww * CT_BK + c];
      if (k < I.K) d.pk[pk_row + k] = s;
    }
    __syncthreads();
  }
  double acc[N_TERMS] = {0, 0, 0, 0, 0, 0, 0, 0};
  acc[T_ZCTG] = obj;
  block_sum(acc);
  write_terms(d.objp, slot0 + blockIdx.x, acc);
}

// ---------------------------------------------------------------------------------------------
// k_adj1: adjoint right-hand side w_i = sum_{m at i} (+-) y_m gF_m, gF_m = dz/df_m summed over
// the contingency tiles (monitored role) and over the rows (outaged role); per-block
// sums of z1 * w for the slack correction.
// ---------------------------------------------------------------------------------------------

template <typename Real, typename Dc>
__global__ void __launch_bounds__(256) k_adj1(Dev<Real, Dc> d, const Blk *__restrict__ blks) {
  const Blk b = blks[blockIdx.x];
  const Inst I = d.inst[b.inst];
  const int t = b.t;
  const int i = b.base + threadIdx.x;
  Dc wz = DcOps<Dc>::zero();
  if (i < I.n) {
    const int ig = I.bus0 + i;
    Dc wsum = DcOps<Dc>::zero();
    for (int e = d.inc_ptr[ig]; e < d.inc_ptr[ig + 1]; ++e) {
      const int code = d.inc[e];
      const int jg = code >> 1;
      const int m = jg - I.br0;
      Real gF = 0;
      for (int kt = 0; kt < I.n_kt; ++kt) gF += d.pm[I.pm0 + ((long long)kt * I.T + t) * I.M + m];
      const int kx = d.br_kidx[jg];
      if (kx >= 0) {
        for (int mt = 0; mt < I.n_mt; ++mt) gF += d.pk[I.pk0 + ((long long)mt * I.T + t) * I.K + kx];
      }
      const Real c = d.br_y[jg] * gF;
      wsum = DcOps<Dc>::add(wsum, DcOps<Dc>::from_real((code & 1) ? -c : c));
    }
    d.w[I.tb0 + (long long)t * I.n + i] = wsum;
    DcOps<Dc>::mac(wz, wsum, d.z1[I.bus0 + i]);
  }
  Dc s = block_sum_dc(wz);
  if (threadIdx.x == 0) d.spart[I.ib0 + (long long)t * I.n_ib + b.ib] = s;
}

// ---------------------------------------------------------------------------------------------
// k_bwd1: adjoints of the four end flows -> adjoints of (v_f, v_o, delta) per branch-period
// ---------------------------------------------------------------------------------------------

template <typename Real, typename Dc>
__global__ void __launch_bounds__(256) k_bwd1(Dev<Real, Dc> d, const Blk *__restrict__ blks, const Real *__restrict__ x) {
  const Blk b = blks[blockIdx.x];
  const Inst I = d.inst[b.inst];
  const int t = b.t;
  const int j = b.base + threadIdx.x;
  if (j >= I.M) return;
  XView<Real> X(x, I);
  const Real dt = d.dt[I.tp0 + t];
  const int jg = I.br0 + j;
  const int f = d.br_from[jg] - I.bus0, o = d.br_to[jg] - I.bus0;
  const long long tb = I.tb0 + (long long)t * I.n;
  const long long e = I.tm0 + (long long)t * I.M + j;
  Real gpf = d.dP[tb + f], gpt = d.dP[tb + o];
  Real gqf = d.dQ[tb + f], gqt = d.dQ[tb + o];
  const Real pf = d.pf[e], qf = d.qf[e], pt = d.pt[e], qt = d.qt[e];
  // thermal (Example 1)
  const Real sf2 = pf * pf + qf * qf, st2 = pt * pt + qt * qt;
  const Real smax = d.br_smax[jg];
  if (fmax(sf2, st2) > smax * smax) {
    const Real sf = dsqrt(sf2), st = dsqrt(st2);
    const bool fr = sf >= st;
    Real val, der;
    soft_relu((fr ? sf : st) - smax, d.eps, val, der);
    const Real k = dt * d.c_s * d.beta * der / (fr ? sf : st);
    if (fr) {
      gpf += k * pf;
      gqf += k * qf;
    } else {
      gpt += k * pt;
      gqt += k * qt;
    }
  }
  // contingency reactive part: dz/dqmax2 summed over outages, routed to the larger-|q| end
  Real gq2 = 0;
  for (int kt = 0; kt < I.n_kt; ++kt) gq2 += d.pq[I.pm0 + ((long long)kt * I.T + t) * I.M + j];
  if (d.qside[e]) gqt += Real(2) * qt * gq2;
  else gqf += Real(2) * qf * gq2;
  // chain rule through the pi-model flows
  const Real vf = X.v[(long long)t * I.n + f], vo = X.v[(long long)t * I.n + o];
  const Real dl = X.th[(long long)t * I.n + f] - X.th[(long long)t * I.n + o];
  Real sn, cs;
  dsincos(dl, &sn, &cs);
  const Real g = d.br_g[jg], bb = d.br_b[jg], bc = d.br_bc[jg];
  const Real vv = vf * vo;
  const Real A = -g * cs - bb * sn;  // p_fr cross coefficient
  const Real B = bb * cs - g * sn;   // q_fr
  const Real C = -g * cs + bb * sn;  // p_to
  const Real D = bb * cs + g * sn;   // q_to
  const Real avf = gpf * (2 * g * vf + A * vo) + gqf * (-2 * bc * vf + B * vo) + gpt * (C * vo) + gqt * (D * vo);
  const Real avo = gpf * (A * vf) + gqf * (B * vf) + gpt * (2 * g * vo + C * vf) + gqt * (-2 * bc * vo + D * vf);
  // d/d delta: dA = g sin - b cos = -B ... written out per flow
  const Real ad = vv * (gpf * (g * sn - bb * cs) + gqf * (-bb * sn - g * cs) + gpt * (g * sn + bb * cs) +
                        gqt * (-bb * sn + g * cs));
  d.avf[e] = avf;
  d.avo[e] = avo;
  d.ad[e] = ad;
}

// ---------------------------------------------------------------------------------------------
// k_bwd2: bus gather of branch-end adjoints into g_v, g_theta (R_BUS); generator gradients and
// the cost / headroom / ramp terms (R_GEN).
// ---------------------------------------------------------------------------------------------

template <typename Real, typename Dc>
__global__ void __launch_bounds__(256) k_bwd2(Dev<Real, Dc> d, const Blk *__restrict__ blks, const Real *__restrict__ x,
                                              int slot0) {
  const Blk b = blks[blockIdx.x];
  const Inst I = d.inst[b.inst];
  const int t = b.t;
  double acc[N_TERMS] = {0, 0, 0, 0, 0, 0, 0, 0};
  XView<Real> X(x, I);
  Real *gx = d.g + I.x0;
  const long long n = I.n, G = I.G, T = I.T;
  if (b.role == R_BUS) {
    const int i = b.base + threadIdx.x;
    if (i < I.n) {
      const int ig = I.bus0 + i;
      const long long tm = I.tm0 + (long long)t * I.M - I.br0;
      Real gv = 0, gth = 0;
      for (int e = d.inc_ptr[ig]; e < d.inc_ptr[ig + 1]; ++e) {
        const int code = d.inc[e];
        const long long k = tm + (code >> 1);
        if (code & 1) {
          gv += d.avo[k];
          gth -= d.ad[k];
        } else {
          gv += d.avf[k];
          gth += d.ad[k];
        }
      }
      gx[t * n + i] = gv;
      gx[T * n + t * n + i] = gth;
    }
  } else if (b.role == R_GEN) {
    const int gl = b.base + threadIdx.x;
    if (gl < I.G) {
      const int gg = I.gen0 + gl;
      const int bus = d.gen_bus[gg] - I.bus0;
      const int zn = d.gen_zone[gg] - I.zone0;
      const Real dt = d.dt[I.tp0 + t];
      const long long k = t * G + gl;
      const Real p = X.p[k], r = X.r[k];
      const Real a = d.gen_a[gg], bl = d.gen_b[gg], cr = d.gen_cr[gg], pmax = d.gen_pmax[gg], ramp = d.gen_ramp[gg];
      const long long tb = I.tb0 + (long long)t * I.n;
      Real gp = dt * (2 * a * p + bl) - d.dP[tb + bus] + DcOps<Dc>::to_real(d.ginj[tb + bus]);
      Real gq = -d.dQ[tb + bus];
      Real gr = dt * cr - d.dZ[I.tz0 + (long long)t * I.Z + zn];
      acc[T_COST] = (double)(dt * (a * p * p + bl * p + cr * r));
      const Real wr = d.rho * d.beta;
      Real val, der;
      soft_relu(p + r - pmax, d.eps, val, der);
      acc[T_ZHEAD] = (double)(wr * val);
      gp += wr * der;
      gr += wr * der;
      if (t >= 1) {
        const Real pp = X.p[k - G];
        const Real lim = ramp * dt;
        Real v1, d1, v2, d2;
        soft_relu(p - pp - lim, d.eps, v1, d1);
        soft_relu(pp - p - lim, d.eps, v2, d2);
        acc[T_ZRAMP] = (double)(wr * (v1 + v2));
        gp += wr * (d1 - d2);
      }
      if (t + 1 < I.T) {
        const Real pn = X.p[k + G];
        const Real lim = ramp * d.dt[I.tp0 + t + 1];
        Real v1, d1, v2, d2;
        soft_relu(pn - p - lim, d.eps, v1, d1);
        soft_relu(p - pn - lim, d.eps, v2, d2);
        gp += wr * (d2 - d1);
      }
      gx[2 * T * n + k] = gp;
      gx[2 * T * n + T * G + k] = gq;
      gx[2 * T * n + 2 * T * G + k] = gr;
    }
  }
  block_sum(acc);
  write_terms(d.objp, slot0 + blockIdx.x, acc);
}

// ---------------------------------------------------------------------------------------------
// k_obj: objective per instance from the block partials (fixed order), plus the closed-form
// soft-ReLU floor of the contingency term.
// ---------------------------------------------------------------------------------------------

template <typename Real, typename Dc>
__global__ void __launch_bounds__(256) k_obj(Dev<Real, Dc> d, const int *__restrict__ slot_inst, int n_slots) {
  const int b = blockIdx.x;
  double acc[N_TERMS] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int s = threadIdx.x; s < n_slots; s += blockDim.x) {
    if (slot_inst[s] != b) continue;
#pragma unroll
    for (int k = 0; k < N_TERMS; ++k) acc[k] += d.objp[(long long)s * N_TERMS + k];
  }
  block_sum(acc);
  if (threadIdx.x == 0) {
    const Inst I = d.inst[b];
    double fl = 0.0;
    for (int t = 0; t < I.T; ++t) fl += (double)d.dt[I.tp0 + t];
    acc[T_ZCTG] += fl * I.wfloor_ctg;
    double tot = 0.0;
    for (int k = 0; k < N_TERMS; ++k) {
      d.terms[b * N_TERMS + k] = acc[k];
      tot += acc[k];
    }
    d.obj[b] = tot;
  }
}

// ---------------------------------------------------------------------------------------------
// projected Adam (Alg. 3); the step counter lives on the device and is advanced by the last block
// ---------------------------------------------------------------------------------------------

__device__ unsigned int g_adam_done = 0;

template <typename Real>
__global__ void __launch_bounds__(256) k_adam(Real *__restrict__ x, Real *__restrict__ m, Real *__restrict__ v,
                                              const Real *__restrict__ g, const Real *__restrict__ lo,
                                              const Real *__restrict__ hi, long long n, long long *step, double lr,
                                              double b1, double b2, double eps, int paper_eps) {
  __shared__ Real sc[2];
  if (threadIdx.x == 0) {
    const double i = (double)(*step + 1);
    sc[0] = (Real)(1.0 / (1.0 - pow(b1, i)));
    sc[1] = (Real)(1.0 / (1.0 - pow(b2, i)));
  }
  __syncthreads();
  const Real c1 = sc[0], c2 = sc[1];
  const Real B1 = (Real)b1, B2 = (Real)b2, E = (Real)eps, LR = (Real)lr;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const Real gk = g[k];
    const Real mk = B1 * m[k] + (Real(1) - B1) * gk;
    const Real vk = B2 * v[k] + (Real(1) - B2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const Real mh = mk * c1, vh = vk * c2;
    const Real num = paper_eps ? mh + E : mh;
    Real xn = x[k] - LR * num / (dsqrt(vh) + E);
    xn = xn < lo[k] ? lo[k] : xn;
    xn = xn > hi[k] ? hi[k] : xn;
    x[k] = xn;
  }
  // last block advances the step counter
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(&g_adam_done, 1u);
    if (prev == gridDim.x - 1) {
      *step += 1;
      g_adam_done = 0;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------

template <typename Real, typename Dc>
size_t ctg_smem_bytes(int T) {
  return sizeof(Real) * ((size_t)T * (3 * CT_BM + CT_BK) + 3 * CT_BM + 8 * CT_BK);
}

// Record a timing event on s; inside stream capture it becomes an external event node.
static inline void mark(cudaEvent_t *ev, int k, cudaStream_t s) {
  if (!ev) return;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
  else cudaEventRecord(ev[k], s);
}

template <typename Real, typename Dc>
cudaError_t launch_eval(const Dev<Real, Dc> &d, const Launch &L, const void *xv, int maxT, cudaEvent_t *ev) {
  const Real *x = static_cast<const Real *>(xv);
  cudaStream_t s = L.stream;
  mark(ev, 0, s);
  k_fwd1<Real, Dc><<<L.n_fwd1, 256, 0, s>>>(d, L.blk_fwd1, x, L.obj_fwd1);
  mark(ev, 1, s);
  k_fwd2<Real, Dc><<<L.n_fwd2, 256, 0, s>>>(d, L.blk_fwd2, x, L.obj_fwd2);
  mark(ev, 2, s);
  k_dc<Real, Dc, false><<<L.n_dct, DC_ROWS * 32, 0, s>>>(d, L.dct);
  mark(ev, 3, s);
  const size_t sm = ctg_smem_bytes<Real, Dc>(maxT);
  if (L.n_ctt > 0) k_ctg<Real, Dc><<<L.n_ctt, 256, sm, s>>>(d, L.ctt, L.obj_ctg, L.lodf_dtype);
  mark(ev, 4, s);
  k_adj1<Real, Dc><<<L.n_adj1, 256, 0, s>>>(d, L.blk_adj1);
  mark(ev, 5, s);
  k_dc<Real, Dc, true><<<L.n_dct, DC_ROWS * 32, 0, s>>>(d, L.dct);
  mark(ev, 6, s);
  k_bwd1<Real, Dc><<<L.n_bwd1, 256, 0, s>>>(d, L.blk_bwd1, x);
  mark(ev, 7, s);
  k_bwd2<Real, Dc><<<L.n_bwd2, 256, 0, s>>>(d, L.blk_bwd2, x, L.obj_bwd2);
  mark(ev, 8, s);
  k_obj<Real, Dc><<<d.n_inst, 256, 0, s>>>(d, L.slot_inst, L.n_obj_slots);
  mark(ev, 9, s);
  return cudaGetLastError();
}

template <typename Real, typename Dc>
cudaError_t prepare_eval(int maxT) {
  const size_t sm = ctg_smem_bytes<Real, Dc>(maxT);
  return cudaFuncSetAttribute(k_ctg<Real, Dc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <typename Real>
cudaError_t launch_adam(Real *x, Real *m, Real *v, const Real *g, const Real *lo, const Real *hi, long long n,
                        long long *step, double lr, double b1, double b2, double eps, int paper_eps,
                        cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  k_adam<Real><<<(int)nb, 256, 0, s>>>(x, m, v, g, lo, hi, n, step, lr, b1, b2, eps, paper_eps);
  return cudaGetLastError();
}

template cudaError_t launch_eval<double, double>(const Dev<double, double> &, const Launch &, const void *, int,
                                                 cudaEvent_t *);
template cudaError_t launch_eval<float, df32>(const Dev<float, df32> &, const Launch &, const void *, int,
                                               cudaEvent_t *);
template cudaError_t prepare_eval<double, double>(int);
template cudaError_t prepare_eval<float, df32>(int);
template cudaError_t launch_adam<double>(double *, double *, double *, const double *, const double *, const double *,
                                         long long, long long *, double, double, double, double, int, cudaStream_t);
template cudaError_t launch_adam<float>(float *, float *, float *, const float *, const float *, const float *,
                                        long long, long long *, double, double, double, double, int, cudaStream_t);

}  // namespace qg
