// Internal declarations shared by the host setup (qg_host.cu) and the device
// kernels (qg_kernels.cu) of libqg.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qg.h"

namespace qg {

// Objective terms, in the order qg_breakdown reports them.
enum Term { T_COST = 0, T_ZP, T_ZQ, T_ZS, T_ZRZ, T_ZHEAD, T_ZRAMP, T_ZCTG, N_TERMS };

// One instance of a batch.  Entity ids inside the kernels are global (offset
// by bus0/br0/gen0/zone0/ctg0); per-period arrays are period-major blocks that
// start at tb0 (T x n), tm0 (T x M), tg0 (T x G), tz0 (T x Z), tp0 (T).
struct Inst {
  int n, M, G, Z, T, K, ref;
  int bus0, br0, gen0, zone0, ctg0, tp0;
  int n_mt, n_kt;          // contingency tiles along monitored branches / outages
  long long x0;            // first variable of this instance
  long long tb0, tm0, tg0, tz0;
  long long z0;            // dense Laplacian inverse, n x n (ref row/col zero)
  long long l0;            // line-outage block, M x K (row m, column k)
  long long pm0, pk0;      // contingency partials: [n_kt][T][M] and [n_mt][T][K]
  long long ib0;           // per-period bus-block partials: [T][n_ib]
  int n_ib;                // bus blocks per period
  double wfloor_ctg;       // c_s * beta * eps * (M*K - K): soft-ReLU floor of the contingency term per hour
  double inv_n;            // 1 / n, and its double-FP32 split
  float inv_n_hi, inv_n_lo;
};

// Block roles of the descriptor-driven kernels.
enum Role : int { R_BRANCH = 0, R_ZONE = 1, R_BUS = 2, R_GEN = 3, R_NONE = 7 };

// One thread block of a descriptor-driven launch: which instance, which period,
// which slice of entities [base, base + blockDim) and what to do.
struct Blk {
  int role;
  int inst;
  int t;
  int base;
  int ib;  // bus-block index within the period (R_BUS)
};

// Tile of the dense DC apply: rows [i0, i0 + rows) of instance inst.
struct DcTile {
  int inst;
  int i0;
};

// Tile of the contingency kernel: monitored rows [m0, m0+BM) x outages [k0, k0+BK).
struct CtgTile {
  int inst;
  int m0, k0;
  int mt, kt;
};

// Double-FP32 value (unevaluated sum hi + lo), used for the FP64-accurate DC
// solves of the mixed path: GB300's FP64 pipe is ~1/60 of its FP32 rate.
struct df32 {
  float hi, lo;
};

// Device-side arrays.  Real is double (QG_FP64) or float (QG_MIXED); Dc is
// double or df32 (the DC-solve value type); Lodf is the line-outage storage type.
template <typename Real, typename Dc>
struct Dev {
  int n_inst;
  const Inst *inst;
  // network (global entity ids)
  const int *br_from, *br_to, *br_kidx;  // kidx: outage index of the branch within its instance, -1 if none
  const Real *br_g, *br_b, *br_bc, *br_smax, *br_sctg, *br_y;  // bc = b + b_ch/2
  const int *gen_bus, *gen_zone;
  const Real *gen_a, *gen_b, *gen_cr, *gen_pmax, *gen_ramp;
  const int *inc_ptr, *inc;           // bus -> (branch << 1 | side), side 1 = "to" end
  const int *bgen_ptr, *bgen;         // bus -> generators
  const int *zgen_ptr, *zgen;         // zone -> generators
  const int *ctg_br;                  // [K total] global branch id of each outage
  const Real *load_p, *load_q;        // [sum T n]
  const Real *rreq;                   // [sum T Z]
  const Real *dt;                     // [sum T]
  const Dc *zinv;                     // [sum n^2]
  const Dc *z1;                       // [sum n] row sums of zinv (global bus id)
  const void *lodf;                   // [sum M K], element type per lodf_dtype
  const Real *lo, *hi;                // Adam clip box [n_x]
  // penalty parameters
  Real c_p, c_q, c_s, c_rz, rho, eps, beta;
  // work buffers
  Real *pf, *qf, *pt, *qt, *qm2;      // [sum T M]
  unsigned char *qside;               // [sum T M] 1 if the "to" end carries the larger |q|
  Real *dP, *dQ;                      // [sum T n]
  Real *dZ;                           // [sum T Z]
  Dc *pinj, *th, *w, *ginj;           // [sum T n]
  Dc *mupart, *spart;                 // [sum T n_ib]
  Real *pm, *pq, *pk;                 // contingency partials
  Real *avf, *avo, *ad;               // branch-end adjoints [sum T M]
  double *objp;                       // [n_obj_slots][N_TERMS]
  double *obj, *terms;                // [n_inst], [n_inst][N_TERMS]
  Real *g;                            // [n_x]
  long long *step;                    // Adam step counter (device)
};

struct Launch {
  cudaStream_t stream;
  // descriptor tables (device) and their sizes
  const Blk *blk_fwd1; int n_fwd1;
  const Blk *blk_fwd2; int n_fwd2;
  const Blk *blk_adj1; int n_adj1;
  const Blk *blk_bwd1; int n_bwd1;
  const Blk *blk_bwd2; int n_bwd2;
  const DcTile *dct; int n_dct;
  const CtgTile *ctt; int n_ctt;
  int obj_fwd1, obj_fwd2, obj_ctg, obj_bwd2;  // first objective slot of each launch
  int n_obj_slots;
  const int *slot_inst;  // instance of every objective slot
  int lodf_dtype;
  long long n_x;
};

template <typename Real, typename Dc>
cudaError_t launch_eval(const Dev<Real, Dc> &d, const Launch &L, const void *x, int maxT, cudaEvent_t *ev);

// Number of timed phases: the nine evaluation kernels and the Adam step.
constexpr int N_PHASES = 10;

template <typename Real, typename Dc>
cudaError_t prepare_eval(int maxT);

template <typename Real>
cudaError_t launch_adam(Real *x, Real *m, Real *v, const Real *g, const Real *lo, const Real *hi, long long n,
                        long long *step, double lr, double b1, double b2, double eps, int paper_eps,
                        cudaStream_t s);


}  // namespace qg
