// FP64 CPU evaluation of the QuasiGrad penalized objective and its gradient, C++17 + OpenMP.
//
// TEST INFRASTRUCTURE ONLY: the timed CPU baseline of the benchmark and its reference arm, and the
// tests that pin it to the numpy oracle (oracle/qg_oracle.py), use it; the library's product path
// never does, and it shares no code, header or layout with the CUDA path.
//
// It computes what oracle/qg_oracle.py computes for cases with plain producers (quadratic costs,
// no bid blocks, consumers, on-status or transformers; others are refused), with its own data
// layout and loop order:
//   * pi-model AC branch flows (sign convention of the Sec. II-F line-flow example), the bus P/Q
//     mismatch of Example 4 and its soft-abs penalty, the thermal penalty on the worse branch end
//     (Example 1), the zonal reserve shortfall, and the headroom and ramp penalties of
//     Eq. nlp_updated, with the generator and reserve costs;
//   * the contingency term of Sec. II-E: base DC solve with the uniform slack (Eqs. Yb_solve,
//     p_flow), the rank-1 correction of each outage (Eq. rank_correct, with the denominator
//     1 - y_k a_k^T Yhat^-1 a_k), the overload penalty (Eqs. sfr_pen-zctg) and the adjoint solve
//     (Eq. 2nd_lin_sys) with the slack correction (Eq. correction).
// The adjoint solves of one period are summed before they are applied: by the same rank-1 identity
// eta_k = Yhat^-1 W_k + u_k y_k (u_k^T W_k) / den_k (u_k = Yhat^-1 a_k, Yhat symmetric), so
// sum_k eta_k = Yhat^-1 (sum_k W_k) + sum_k u_k y_k (u_k^T W_k) / den_k: one solve per period
// instead of one per outage, the same sum.  Yhat^-1 is an explicit inverse (Cholesky, dense grids).
//
// Work is split into (period, block of outages) tasks for OpenMP; each task writes its own partial
// sums, added afterwards in task order, so the result does not depend on the thread count.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

struct qgo_case {
  int32_t n, M, G, Z, T, K, ref;
  const int32_t *br_from, *br_to;                 // [M]
  const double *br_r, *br_x, *br_b;               // [M] series r, x and total charging b
  const double *s_max, *s_max_ctg;                // [M] ratings (base case, post-contingency)
  const int32_t *gen_bus, *gen_zone;              // [G]
  const double *cost_a, *cost_b, *cost_r;         // [G]
  const double *pmax, *ramp;                      // [G]
  const double *dt;                               // [T] period lengths (hours)
  const double *load_p, *load_q;                  // [T][n]
  const double *reserve_req;                      // [T][Z]
  const int32_t *ctg;                             // [K] outaged branch ids
  double c_p, c_q, c_s, c_rz, rho, eps, beta;
};

}  // extern "C"

namespace {

constexpr int KBLOCK = 32;  // outages per task

double soft_abs(double x, double eps) { return std::sqrt(x * x + eps * eps); }
double soft_abs_grad(double x, double eps) {
  const double s = std::sqrt(x * x + eps * eps);
  return s > 0 ? x / s : 0.0;
}
double soft_relu(double x, double eps) {
  const double m = x > 0 ? x : 0.0;
  return std::sqrt(m * m + eps * eps);
}
double soft_relu_grad(double x, double eps) {
  const double m = x > 0 ? x : 0.0;
  const double s = std::sqrt(m * m + eps * eps);
  return s > 0 ? m / s : 0.0;
}

struct Oracle {
  // the case (copied)
  int n, M, G, Z, T, K, ref;
  std::vector<int> f, o, gbus, gzone, ctg;
  std::vector<double> g, b, bch, smax, sctg, ca, cb, cr, pmax, ramp, dt, lp, lq, req;
  double c_p, c_q, c_s, c_rz, rho, eps, beta;
  // DC set-up: y = -b_sr, inverse of the reduced Laplacian (full n x n, zero row and column at the
  // reference bus), u_k = Yhat^-1 a_k as full-length vectors, the rank-1 denominators
  std::vector<double> y, Yinv, U, den;
};

// Cholesky factorization and inverse of the SPD matrix A (m x m, row-major), in place.
bool spd_inverse(std::vector<double> &A, int m) {
  std::vector<double> L(A);
  for (int j = 0; j < m; ++j) {
    double d = L[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    L[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double s = L[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      L[(size_t)i * m + j] = s / d;
    }
  }
  // columns of the inverse: solve L L^T x = e_c
#pragma omp parallel for schedule(dynamic, 8)
  for (int c = 0; c < m; ++c) {
    std::vector<double> z(m, 0.0);
    for (int i = c; i < m; ++i) {  // forward: L z = e_c (z_i = 0 for i < c)
      double s = i == c ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= L[(size_t)i * m + k] * z[k];
      z[i] = s / L[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {  // backward: L^T x = z
      double s = z[i];
      for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * z[k];
      z[i] = s / L[(size_t)i * m + i];
    }
    for (int i = 0; i < m; ++i) A[(size_t)i * m + c] = z[i];
  }
  return true;
}

}  // namespace

extern "C" {

// Copies the case and builds the DC set-up; NULL when the case is outside this evaluation's scope
// (the numpy oracle covers it) or the reduced Laplacian is not positive definite.
void *qgo_prepare(const qgo_case *c) {
  if (!c || c->n < 2 || c->M < 1 || c->T < 1 || c->G < 0 || c->Z < 1 || c->K < 0) return nullptr;
  Oracle *h = new Oracle();
  h->n = c->n; h->M = c->M; h->G = c->G; h->Z = c->Z; h->T = c->T; h->K = c->K; h->ref = c->ref;
  const int n = c->n, M = c->M, G = c->G, T = c->T, K = c->K;
  h->f.assign(c->br_from, c->br_from + M);
  h->o.assign(c->br_to, c->br_to + M);
  h->gbus.assign(c->gen_bus, c->gen_bus + G);
  h->gzone.assign(c->gen_zone, c->gen_zone + G);
  h->ctg.assign(c->ctg, c->ctg + K);
  h->g.resize(M); h->b.resize(M); h->y.resize(M);
  for (int m = 0; m < M; ++m) {  // g + j b = 1 / (r + j x); y = x / (r^2 + x^2) = -b
    const double den = c->br_r[m] * c->br_r[m] + c->br_x[m] * c->br_x[m];
    h->g[m] = c->br_r[m] / den;
    h->b[m] = -c->br_x[m] / den;
    h->y[m] = c->br_x[m] / den;
  }
  h->bch.assign(c->br_b, c->br_b + M);
  h->smax.assign(c->s_max, c->s_max + M);
  h->sctg.assign(c->s_max_ctg, c->s_max_ctg + M);
  h->ca.assign(c->cost_a, c->cost_a + G);
  h->cb.assign(c->cost_b, c->cost_b + G);
  h->cr.assign(c->cost_r, c->cost_r + G);
  h->pmax.assign(c->pmax, c->pmax + G);
  h->ramp.assign(c->ramp, c->ramp + G);
  h->dt.assign(c->dt, c->dt + T);
  h->lp.assign(c->load_p, c->load_p + (size_t)T * n);
  h->lq.assign(c->load_q, c->load_q + (size_t)T * n);
  h->req.assign(c->reserve_req, c->reserve_req + (size_t)T * c->Z);
  h->c_p = c->c_p; h->c_q = c->c_q; h->c_s = c->c_s; h->c_rz = c->c_rz; h->rho = c->rho; h->eps = c->eps;
  h->beta = c->beta;
  // reduced Laplacian Yhat = E_hat^T diag(y) E_hat over the buses other than the reference
  std::vector<int> red(n, -1);
  int m1 = 0;
  for (int i = 0; i < n; ++i)
    if (i != c->ref) red[i] = m1++;
  std::vector<double> Y((size_t)m1 * m1, 0.0);
  for (int m = 0; m < M; ++m) {
    const int a = red[h->f[m]], bb = red[h->o[m]];
    if (a >= 0) Y[(size_t)a * m1 + a] += h->y[m];
    if (bb >= 0) Y[(size_t)bb * m1 + bb] += h->y[m];
    if (a >= 0 && bb >= 0) {
      Y[(size_t)a * m1 + bb] -= h->y[m];
      Y[(size_t)bb * m1 + a] -= h->y[m];
    }
  }
  if (!spd_inverse(Y, m1)) {
    delete h;
    return nullptr;
  }
  h->Yinv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (red[i] >= 0 && red[j] >= 0) h->Yinv[(size_t)i * n + j] = Y[(size_t)red[i] * m1 + red[j]];
  // u_k = Yhat^-1 a_k (a_k: +1 at the from bus, -1 at the to bus), den_k = 1 - y_k a_k^T u_k
  h->U.assign((size_t)K * n, 0.0);
  h->den.assign(K, 0.0);
  for (int k = 0; k < K; ++k) {
    const int j = h->ctg[k], a = h->f[j], bb = h->o[j];
    double *u = &h->U[(size_t)k * n];
    for (int i = 0; i < n; ++i) u[i] = h->Yinv[(size_t)i * n + a] - h->Yinv[(size_t)i * n + bb];
    h->den[k] = 1.0 - h->y[j] * (u[a] - u[bb]);
  }
  return h;
}

void qgo_free(void *p) { delete static_cast<Oracle *>(p); }

// Phi(x) with terms[8] = (cost, z_p, z_q, z_s, z_rz, z_headroom, z_ramp, z_ctg) and, when grad is
// not NULL, its gradient; x and grad in the layout [v | theta | p | q | r], each block T rows
// (period-major).  threads <= 0: OpenMP's default.  Returns Phi.
double qgo_eval(void *ph, const double *x, double *grad, double *terms, int32_t threads) {
  const Oracle &h = *static_cast<Oracle *>(ph);
  const int n = h.n, M = h.M, G = h.G, Z = h.Z, T = h.T, K = h.K;
  if (threads > 0) omp_set_num_threads(threads);
  const double *V = x, *TH = x + (size_t)T * n, *P = x + 2 * (size_t)T * n, *Qg = P + (size_t)T * G,
               *R = Qg + (size_t)T * G;
  std::vector<double> gv((size_t)T * n, 0.0), gth((size_t)T * n, 0.0), gp((size_t)T * G, 0.0),
      gq((size_t)T * G, 0.0), gr((size_t)T * G, 0.0);
  // per-period partial terms (summed in period order at the end)
  std::vector<double> tcost(T, 0.0), tzp(T, 0.0), tzq(T, 0.0), tzs(T, 0.0), tzrz(T, 0.0), thead(T, 0.0),
      tramp(T, 0.0);
  // AC quantities kept for the contingency stage and the pull-back
  std::vector<double> pf((size_t)T * M), qf((size_t)T * M), pt((size_t)T * M), qt((size_t)T * M);
  std::vector<double> g_pf((size_t)T * M), g_qf((size_t)T * M), g_pt((size_t)T * M), g_qt((size_t)T * M);
  std::vector<double> qmax2((size_t)T * M), fbase((size_t)T * M);
  std::vector<char> use_qf((size_t)T * M);
  const double eps = h.eps, beta = h.beta;

#pragma omp parallel for schedule(static)
  for (int t = 0; t < T; ++t) {
    const double *v = V + (size_t)t * n, *th = TH + (size_t)t * n, *p = P + (size_t)t * G, *q = Qg + (size_t)t * G,
                 *r = R + (size_t)t * G;
    double *gpt = gp.data() + (size_t)t * G, *gqt = gq.data() + (size_t)t * G, *grt = gr.data() + (size_t)t * G;
    const double d = h.dt[t];
    // costs
    double cost = 0.0;
    for (int k = 0; k < G; ++k) {
      cost += d * (h.ca[k] * p[k] * p[k] + h.cb[k] * p[k] + h.cr[k] * r[k]);
      gpt[k] += d * (2 * h.ca[k] * p[k] + h.cb[k]);
      grt[k] += d * h.cr[k];
    }
    tcost[t] = cost;
    // pi-model flows and the bus mismatch
    std::vector<double> Pb(h.lp.begin() + (size_t)t * n, h.lp.begin() + (size_t)(t + 1) * n);
    std::vector<double> Qb(h.lq.begin() + (size_t)t * n, h.lq.begin() + (size_t)(t + 1) * n);
    for (int m = 0; m < M; ++m) {
      const int a = h.f[m], bb = h.o[m];
      const double dl = th[a] - th[bb], c = std::cos(dl), s = std::sin(dl);
      const double vv = v[a] * v[bb], gm = h.g[m], bm = h.b[m], bc = h.bch[m] / 2;
      const size_t e = (size_t)t * M + m;
      pf[e] = gm * v[a] * v[a] + (-gm * c - bm * s) * vv;
      qf[e] = -(bm + bc) * v[a] * v[a] + (bm * c - gm * s) * vv;
      pt[e] = gm * v[bb] * v[bb] + (-gm * c + bm * s) * vv;
      qt[e] = -(bm + bc) * v[bb] * v[bb] + (bm * c + gm * s) * vv;
      Pb[a] += pf[e]; Pb[bb] += pt[e];
      Qb[a] += qf[e]; Qb[bb] += qt[e];
    }
    for (int k = 0; k < G; ++k) {
      Pb[h.gbus[k]] -= p[k];
      Qb[h.gbus[k]] -= q[k];
    }
    const double wp = d * h.c_p * beta, wq = d * h.c_q * beta;
    std::vector<double> dP(n), dQ(n);
    double zp = 0.0, zq = 0.0;
    for (int i = 0; i < n; ++i) {
      zp += wp * soft_abs(Pb[i], eps);
      zq += wq * soft_abs(Qb[i], eps);
      dP[i] = wp * soft_abs_grad(Pb[i], eps);
      dQ[i] = wq * soft_abs_grad(Qb[i], eps);
    }
    tzp[t] = zp;
    tzq[t] = zq;
    for (int k = 0; k < G; ++k) {
      gpt[k] -= dP[h.gbus[k]];
      gqt[k] -= dQ[h.gbus[k]];
    }
    // thermal limit on the worse end (ties to the from end)
    const double ws = d * h.c_s * beta;
    double zs = 0.0;
    for (int m = 0; m < M; ++m) {
      const size_t e = (size_t)t * M + m;
      g_pf[e] = dP[h.f[m]];
      g_pt[e] = dP[h.o[m]];
      g_qf[e] = dQ[h.f[m]];
      g_qt[e] = dQ[h.o[m]];
      const double sf = std::sqrt(pf[e] * pf[e] + qf[e] * qf[e]), st = std::sqrt(pt[e] * pt[e] + qt[e] * qt[e]);
      const bool fr = sf >= st;
      const double u = (fr ? sf : st) - h.smax[m];
      zs += ws * soft_relu(u, eps);
      const double dS = ws * soft_relu_grad(u, eps);
      if (fr && sf > 0) {
        g_pf[e] += dS / sf * pf[e];
        g_qf[e] += dS / sf * qf[e];
      } else if (!fr && st > 0) {
        g_pt[e] += dS / st * pt[e];
        g_qt[e] += dS / st * qt[e];
      }
      // the reactive part of the post-contingency rating test: q of the worse end (ties to from)
      use_qf[e] = qf[e] * qf[e] >= qt[e] * qt[e];
      qmax2[e] = use_qf[e] ? qf[e] * qf[e] : qt[e] * qt[e];
    }
    tzs[t] = zs;
    // zonal reserve shortfall
    std::vector<double> rz(Z, 0.0);
    for (int k = 0; k < G; ++k) rz[h.gzone[k]] += r[k];
    const double wz = d * h.c_rz * beta;
    double zrz = 0.0;
    for (int zz = 0; zz < Z; ++zz) {
      const double u = h.req[(size_t)t * Z + zz] - rz[zz];
      zrz += wz * soft_relu(u, eps);
      rz[zz] = wz * soft_relu_grad(u, eps);  // now the derivative
    }
    tzrz[t] = zrz;
    for (int k = 0; k < G; ++k) grt[k] -= rz[h.gzone[k]];
    // headroom p + r <= pmax
    const double wr = h.rho * beta;
    double zh = 0.0;
    for (int k = 0; k < G; ++k) {
      const double u = p[k] + r[k] - h.pmax[k];
      zh += wr * soft_relu(u, eps);
      const double dH = wr * soft_relu_grad(u, eps);
      gpt[k] += dH;
      grt[k] += dH;
    }
    thead[t] = zh;
    // base DC flows: injections with the uniform slack, theta = Yhat^-1 pbar, f = y (theta_f - theta_o)
    std::vector<double> inj(n);
    for (int i = 0; i < n; ++i) inj[i] = -h.lp[(size_t)t * n + i];
    for (int k = 0; k < G; ++k) inj[h.gbus[k]] += p[k];
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += inj[i];
    mean /= n;
    for (int i = 0; i < n; ++i) inj[i] -= mean;
    std::vector<double> thd(n, 0.0);
    for (int i = 0; i < n; ++i) {
      const double *row = &h.Yinv[(size_t)i * n];
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += row[j] * inj[j];
      thd[i] = s;
    }
    for (int m = 0; m < M; ++m) fbase[(size_t)t * M + m] = h.y[m] * (thd[h.f[m]] - thd[h.o[m]]);
  }

  // ramps (couple consecutive periods; serial)
  for (int t = 1; t < T; ++t) {
    const double wr = h.rho * beta;
    double zr = 0.0;
    for (int k = 0; k < G; ++k) {
      const double lim = h.ramp[k] * h.dt[t];
      const double dp = P[(size_t)t * G + k] - P[(size_t)(t - 1) * G + k];
      zr += wr * (soft_relu(dp - lim, eps) + soft_relu(-dp - lim, eps));
      const double dU = wr * soft_relu_grad(dp - lim, eps), dD = wr * soft_relu_grad(-dp - lim, eps);
      gp[(size_t)t * G + k] += dU - dD;
      gp[(size_t)(t - 1) * G + k] += dD - dU;
    }
    tramp[t] = zr;
  }

  // contingencies: tasks (period, block of KBLOCK outages), each with its own partial sums
  const int nkb = (K + KBLOCK - 1) / KBLOCK, ntask = T * nkb;
  std::vector<double> tz(ntask, 0.0), tq2((size_t)ntask * M, 0.0), tW((size_t)ntask * n, 0.0),
      tV((size_t)ntask * n, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int task = 0; task < ntask; ++task) {
    const int t = task / nkb, k0 = (task % nkb) * KBLOCK, k1 = std::min(K, k0 + KBLOCK);
    const double *f = &fbase[(size_t)t * M], *q2 = &qmax2[(size_t)t * M];
    double *gq2 = &tq2[(size_t)task * M], *W = &tW[(size_t)task * n], *Vs = &tV[(size_t)task * n];
    const double w = h.dt[t] * h.c_s * beta;
    std::vector<double> Wk(n);
    double z = 0.0;
    for (int k = k0; k < k1; ++k) {
      const int j = h.ctg[k];
      const double *u = &h.U[(size_t)k * n];
      const double sk = f[j] / h.den[k];  // theta_k = theta + u_k f_k / den_k (Eq. rank_correct)
      std::fill(Wk.begin(), Wk.end(), 0.0);
      double uW = 0.0;  // u_k^T W_k
      for (int m = 0; m < M; ++m) {
        if (m == j) continue;  // the outaged branch carries nothing and is not monitored
        const int a = h.f[m], bb = h.o[m];
        const double Pm = f[m] + h.y[m] * sk * (u[a] - u[bb]);
        const double s = std::sqrt(Pm * Pm + q2[m]), du = s - h.sctg[m];
        z += w * soft_relu(du, eps);
        const double dsig = w * soft_relu_grad(du, eps);
        if (dsig == 0.0 || !(s > 0)) continue;
        gq2[m] += dsig * 0.5 / s;
        const double yD = h.y[m] * dsig * Pm / s;  // y_m dz/dp_m
        Wk[a] += yD;
        Wk[bb] -= yD;
        uW += yD * (u[a] - u[bb]);
      }
      for (int i = 0; i < n; ++i) W[i] += Wk[i];
      const double ck = h.y[j] * uW / h.den[k];
      for (int i = 0; i < n; ++i) Vs[i] += ck * u[i];
    }
    tz[task] = z;
  }
  // per period: eta = Yhat^-1 (sum W) + sum u_k c_k, slack correction, pull-back to p and q
  std::vector<double> tzc(T, 0.0);
#pragma omp parallel for schedule(static)
  for (int t = 0; t < T; ++t) {
    std::vector<double> W(n, 0.0), eta(n, 0.0), q2g(M, 0.0);
    double z = 0.0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int task = t * nkb + kb;
      z += tz[task];
      for (int i = 0; i < n; ++i) {
        W[i] += tW[(size_t)task * n + i];
        eta[i] += tV[(size_t)task * n + i];
      }
      for (int m = 0; m < M; ++m) q2g[m] += tq2[(size_t)task * M + m];
    }
    tzc[t] = z;
    W[h.ref] = 0.0;  // the reference bus is not in the reduced system
    for (int i = 0; i < n; ++i) {
      const double *row = &h.Yinv[(size_t)i * n];
      double s = 0.0;
      for (int jj = 0; jj < n; ++jj) s += row[jj] * W[jj];
      eta[i] += s;
    }
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += eta[i];
    mean /= n;
    for (int k = 0; k < G; ++k) gp[(size_t)t * G + k] += eta[h.gbus[k]] - mean;
    for (int m = 0; m < M; ++m) {
      const size_t e = (size_t)t * M + m;
      if (use_qf[e]) g_qf[e] += 2 * qf[e] * q2g[m];
      else g_qt[e] += 2 * qt[e] * q2g[m];
    }
  }

  // branch-end adjoints back to (v, theta), per period (each period owns its rows of gv, gth)
#pragma omp parallel for schedule(static)
  for (int t = 0; t < T; ++t) {
    const double *v = V + (size_t)t * n, *th = TH + (size_t)t * n;
    double *gvt = gv.data() + (size_t)t * n, *gtht = gth.data() + (size_t)t * n;
    for (int m = 0; m < M; ++m) {
      const int a = h.f[m], bb = h.o[m];
      const size_t e = (size_t)t * M + m;
      const double dl = th[a] - th[bb], c = std::cos(dl), s = std::sin(dl);
      const double gm = h.g[m], bm = h.b[m], bc = h.bch[m] / 2, vf = v[a], vo = v[bb], vv = vf * vo;
      const double Gpf = g_pf[e], Gqf = g_qf[e], Gpt = g_pt[e], Gqt = g_qt[e];
      gvt[a] += Gpf * (2 * gm * vf + (-gm * c - bm * s) * vo) + Gqf * (-2 * (bm + bc) * vf + (bm * c - gm * s) * vo) +
                Gpt * ((-gm * c + bm * s) * vo) + Gqt * ((bm * c + gm * s) * vo);
      gvt[bb] += Gpf * ((-gm * c - bm * s) * vf) + Gqf * ((bm * c - gm * s) * vf) +
                 Gpt * (2 * gm * vo + (-gm * c + bm * s) * vf) + Gqt * (-2 * (bm + bc) * vo + (bm * c + gm * s) * vf);
      const double gd = Gpf * ((gm * s - bm * c) * vv) + Gqf * ((-bm * s - gm * c) * vv) + Gpt * ((gm * s + bm * c) * vv) +
                        Gqt * ((-bm * s + gm * c) * vv);
      gtht[a] += gd;
      gtht[bb] -= gd;
    }
  }

  double tt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    tt[0] += tcost[t]; tt[1] += tzp[t]; tt[2] += tzq[t]; tt[3] += tzs[t];
    tt[4] += tzrz[t]; tt[5] += thead[t]; tt[6] += tramp[t]; tt[7] += tzc[t];
  }
  double obj = 0.0;
  for (int k = 0; k < 8; ++k) {
    obj += tt[k];
    if (terms) terms[k] = tt[k];
  }
  if (grad) {
    double *o = grad;
    std::memcpy(o, gv.data(), sizeof(double) * gv.size()); o += gv.size();
    std::memcpy(o, gth.data(), sizeof(double) * gth.size()); o += gth.size();
    std::memcpy(o, gp.data(), sizeof(double) * gp.size()); o += gp.size();
    std::memcpy(o, gq.data(), sizeof(double) * gq.size()); o += gq.size();
    std::memcpy(o, gr.data(), sizeof(double) * gr.size());
  }
  return obj;
}

int32_t qgo_max_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
