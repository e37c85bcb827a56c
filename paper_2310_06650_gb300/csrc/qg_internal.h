// Internal declarations shared by the host set-up (qg_host.cu) and the device
// kernels (qg_kernels.cu) of libqg.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only NVTX v3: a no-op unless a profiler injects itself

#include "../../include/qg.h"

namespace qg {
// A named NVTX range over a scope (a stage launch, a public call), visible on a profiler's timeline.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace qg

namespace qg {

// Objective terms, in the order qg_breakdown reports them.
enum Term { T_COST = 0, T_ZP, T_ZQ, T_ZS, T_ZRZ, T_ZHEAD, T_ZRAMP, T_ZCTG, N_TERMS };

constexpr int MAXB = 32;       // instances per handle (the instance table travels as a kernel parameter)
constexpr int MAXSPAN = 192;   // block spans per launch
constexpr int NTHR = 256;      // threads per block of every stage kernel
constexpr int CT_BM = 64, CT_BK = 64;  // contingency tile: monitored branches x outages
constexpr int DCF_BM = 32, DCF_TC = 8; // forward DC tile: 32 branches x 8 periods
constexpr int PACK = 32;               // CSR entries per warp pack (rows never straddle packs)
constexpr int PACKS_PER_BLOCK = NTHR / 32;
constexpr int S4_PACKS = 2;            // branch-end CSR packs per warp in the bus gather of stage 4, at most
constexpr int S3_SPLIT_MAX = 4;        // threads per branch-period in stage 3 (InstTab::s3q), at most

// One instance of a batch.  Entity ids inside the kernels are global (offset by
// bus0 / br0 / gen0 / zone0 / ctg0 / gb0); per-period arrays are period-major
// blocks starting at tb0 (T x n), tm0 (T x M), tg0 (T x G), tz0 (T x Z), tk0
// (T x K) and tp0 (T).
struct Inst {
  int n, M, G, Z, T, K, Gb;
  int Kp;                // row stride of the line-outage block: K rounded up to a multiple of 4
  int X, xf0;            // transformers; first global transformer id
  int Gc;                // columns of the dense DC products: generator buses, then (dense mode)
                         // one column per transformer (its phase-shift flow)
  int bus0, br0, gen0, zone0, ctg0, gb0, tp0;
  int n_mt, n_kt;        // contingency tiles along monitored branches / outages
  int ctg_mg, n_mg;      // monitored-branch tiles per contingency block, and the number of such groups
  int ctg_tb, ctg_ntc;   // periods per contingency block, and the number of period chunks
  int n_sb;              // stage-3 branch blocks per period (NTHR / InstTab::s3q branches each)
  int s4p;               // branch-end CSR packs per warp in stage 4 (1 or S4_PACKS)
  int bal0, n_bal_pack;  // first entry / number of warp packs of the balance CSR
  int bus_tc;            // periods per stage-2 bus-balance block (several on large plans)
  int adj0, n_adj_pack;  // same for the branch-end adjoint CSR
  long long x0;          // first variable of this instance
  long long tb0, tm0, tg0, tz0, tk0;
  long long pg0;         // PTDF restricted to generator buses: M x Gb, row m
  long long l0;          // line-outage block, M x Kp, row m
  long long pm0, pk0;    // contingency partials: [n_kt][T][M] and [n_mg][T][K]
  long long pf0;         // flags of the row partials: [n_kt][T][n_mt], 1 where a 64-row tile has any
  long long lm0;         // bound-test row maxima of the line-outage block: [n_kt 4][n_mt 64]
  long long rm0;         // clearance minima per chunk of 8 periods (on-demand path): [ctg_ntc NCH][n_mt 64]
                         // with NCH = ceil(ctg_tb / 8), inside T n_mt 64 floats
  int ctg_bound;         // 1: stage 2 bounds each (warp, chunk of periods) before its element screen
  int ctg_lazy;          // 1: on-demand path: the bound tests of a batch of tiles come first, from the
                         // clearance minima of k_ctg_margin; only tiles where some warp fails are
                         // staged, and only failing warps load their piece of the line-outage tile
  long long gi0;         // adjoint DC products of the sparse mode: [T][Gc + 1] (generator buses,
                         // transformers, then n mean(eta))
  long long tx0;         // per-period transformer arrays: [T][X]
  long long xtau0;       // first tau variable (x0 + T (2n + 3G)); phi follow after T X
  long long xu0;         // first on-status variable (after phi; meaningful when uc)
  int uc;                // 1: on-status variables u with startup / shutdown costs (Example 2)
  double inv_n;          // 1 / n
  double hours;          // sum of dt
  double nfloor_ctg;     // M K - K: elements whose soft-ReLU floor eps the contingency term adds in closed form
  int obj_lo, obj_n;     // this instance's stage-1/2 objective slots
  int gen_first, gen_nb; // its device blocks (R_GBUS in stage 4, or R_GEN in stage 5 of the sparse mode):
                         // first block in their launch, count
  int gen_pb;            // (period, device) pairs per device block (the first gen_pb threads)
  int gen_slot0;         // first reduction slot of those blocks (after the stage-1/2 slots)
  int fold_nb, fold_slot0; // its stage-3 fold blocks (each sums up to NTHR stage-1/2 slots) and their
                           // first slot (after the device-block slots)
};

// Roles of the blocks of the fused stage kernels.  R_DCF is the dense forward DC product and R_GBUS
// the dense adjoint product with the device updates at each generator bus; R_SDCF / R_SDCA are their
// counterparts around the sparse-factor solves (flows from the solved angles; right-hand side of
// the adjoint solve), whose device updates are R_GEN / R_XF blocks of stage 5.
enum Role : int { R_BRANCH = 0, R_ZONE, R_DCF, R_BUS, R_CTG, R_GBUS, R_GEN, R_SDCF, R_SDCA, R_XF, R_OBJ };

constexpr int SP_RB = 64;   // dense tail product: rows per block
constexpr int SP_BK = 32;   // dense tail product: columns per shared-memory chunk
constexpr int SP_TMAX = 48; // periods per pass of the dense tail product (16 lanes x 3)

// A run of blocks with one role for one instance: blocks [first, first + per_t * nt);
// block b of the span has period (or period chunk) (b - first) / per_t and slice (b - first) % per_t.
struct Span {
  int first, per_t, nt, inst, role;
};

struct Spans {
  Span s[MAXSPAN];
  int n;
  int n_blocks;
};

struct InstTab {
  Inst I[MAXB];
  int n_inst;
  int fuse;  // 1: stage 4's warps update the devices (the last stage); 0: stage 5 does
  int s3q;   // threads per branch-period in stage 3 (1 or S3_SPLIT_MAX; the kernel's template argument)
};

// Double-FP32 value (unevaluated sum hi + lo) carrying the FP64-accurate DC
// products of the mixed path: GB300's FP64 pipe runs at ~1/60 of its FP32 rate.
struct df32 {
  float hi, lo;
};

// Device arrays.  Real is double (QG_FP64) or float (QG_MIXED); Dc is the DC
// product type: double, or df32 in the mixed path.
template <typename Real, typename Dc>
struct Dev {
  // network (global ids)
  const int2 *br_end;                 // [sum M] (from, to) bus ids local to the instance
  const int *br_kidx;                 // [sum M] outage index of the branch within its instance, -1 if none
  const Real *br_g, *br_b, *br_hch, *br_smax, *br_s2ctg;  // g_sr, b_sr, b_ch / 2, s_max, s_ctg^2
  const int *gen_bus, *gen_zone, *gen_gb;                 // local bus, local zone, local generator-bus index
  const Real *gen_a, *gen_b, *gen_cr, *gen_pmax;
  const Real *gen_sgn;                // +1 producer, -1 consumer (sign of p, q as supply)
  const Real *gen_pmin, *gen_qmin, *gen_qmax;             // limits scaled by u (commitment)
  const Real *gen_con, *gen_csu, *gen_csd, *gen_uinit;    // on / startup / shutdown cost, u before period 0
  // FP64 copies of the limits the penalized linear constraints subtract (Eq. nlp_updated; Example 2's
  // u-scaled limits) and of the zonal requirements: both paths form those residuals in FP64.  At a
  // solution the constraints are active, so each residual cancels O(1) terms, and the soft-ReLU's
  // derivative moves by 1/eps per unit of residual error.
  const double *lim_pmax, *lim_pmin, *lim_qmin, *lim_qmax, *lim_ramp;  // [sum G]
  const double *lim_rreq;             // [sum T Z]
  const double *lim_dt;               // [sum T]
  const int *blk_ptr;                 // [sum G + 1] bid blocks of each device (Example 3); none: quadratic cost
  const Real *blk_c, *blk_lo, *blk_w; // block price, cumulative start P_{l-1}, width
  const int *gb_ptr, *gb_gen;         // generator bus -> generators: one CSR over the batch's generator buses
  const int *gb_dev0, *gb_ndev;       // [sum Gb] each generator bus's first device (global id) and count
  const int *zgen_ptr, *zgen;         // zone -> generators: one CSR over the batch's zones (global ids)
  const int *ctg_br;                  // [sum K] local branch id of each outage
  const int *br_xf;                   // [sum M] local transformer index of each branch, -1 for lines
  const int *xf_br;                   // [sum X] local branch id of each transformer
  const int *bal_code, *bal_row;      // balance CSR packs: code = j<<2|kind (0 from-end, 1 to-end, 2 generator, 3 pad)
  const int *adj_code, *adj_row;      // branch-end CSR packs (kind 0 / 1 / 3)
  const Real *load_p, *load_q;        // [sum T n]
  const Real *dt;                     // [sum T]
  const Dc *ltot;                     // [sum T] total load per period
  const Dc *load_dc;                  // [T n] active load in the DC product type (sparse mode)
  const Dc *ptdfg;                    // [sum M Gb] PTDF columns of generator buses, row m
  const Dc *ptdfaT;                   // [sum Gc M] adjoint columns, row c: PTDF[m, gb] - (PTDF 1)[m] / n for a
                                      // generator bus (the slack's mean folded in), PSDF[m, x] for a transformer
  const Dc *cload;                    // [sum T M] PTDF * load_t
  const Dc *rsum;                     // [sum M] PTDF * 1
  const void *lodf;                   // [sum M Kp]: float / bf16 / bf16x2 (mixed) or float screening copy
                                      // (FP64); NaN at pads and at each outage's own branch
  const double *lodf64;               // [sum M Kp] FP64 path only
  float *ctg_rmin;                    // per instance at rm0: clearance minima of k_ctg_margin (on-demand path)
  const float *lmax;                  // per instance at lm0, [n_kt 4][n_mt 64]: the largest |L[m, k]| over each
                                      // group of 16 outage columns (as the stage-2 screen reads L; NaN
                                      // ignored), 0 on pad rows; the bound test of the contingency screen
  const Real *lo, *hi;                // clip box [n_x]
  // sparse DC mode (one instance): node positions = eliminated nodes in elimination order, then
  // the tail nodes whose Schur complement S is held through its inverse; node-major work arrays
  // [position][T].  Yhat^-1 b = (forward gather, D_S^-1, S^-1, backward gather), see qg_sparse.h.
  int sp;                             // 1: DC solves through the sparse factor (no PTDF)
  int nr, nS, nT;                     // reduced nodes (n - 1), eliminated nodes, tail nodes
  int n_pchunk;                       // position chunks of 32 (adjoint right-hand-side blocks)
  int n_adj_rows;                     // eliminated positions that are generator buses
  const int *bus_pos;                 // [n] position of each bus, -1 at the reference bus
  const int *pos_gb;                  // [nr] generator-bus index at each position, -1 if none
  const int *pos_bus;                 // [nr] bus at each position
  const int *fw_ptr, *fw_col;         // forward gather rows [nr + 1] / entries (positions)
  const Dc *fw_val;
  const int *bw_ptr, *bw_col;         // backward gather rows [nS + 1] / entries (positions)
  const Dc *bw_val;
  const int *adj_rows;                // [n_adj_rows]
  const Dc *dinv;                     // [nS] 1 / D_S
  const Dc *sinv;                     // [nT nT] S^-1, row-major
  const Dc *z1;                       // [nr] Yhat^-1 1 at each position
  const int *inc_ptr, *inc_code;      // position -> incident branches, code = j << 1 | (1 at the to-end)
  const Dc *ydc;                      // [M] y_j = -b_sr
  Dc *sp_rhs, *sp_u, *sp_th, *sp_zt;  // [nr T], [nr T], [nr T], [nT T]
  Dc *sp_mu;                          // [T] mean injection (uniform slack)
  Dc *sp_part;                        // [n_pchunk][T] partial sums of z1 . w
  Dc *sp_tpart;                       // [tail splits][nT][T] partial sums of the dense tail product
  unsigned int *sp_tick;              // [tail row tiles] last-split tickets (zero between launches)
  // penalty parameters
  Real c_p, c_q, c_s, c_rz, rho, eps, beta;
  double c_s64, eps64, beta64;        // the same options in FP64 (closed-form objective floor)
  int lodf_dtype;
  // work buffers
  Real *pf, *qf, *pt, *qt, *qm2;      // [sum T M]
  unsigned char *qside;               // [sum T M] 1 if the "to" end carries the larger |q|
  Real *fre;                          // [sum T M] base DC flows
  float *f32;                         // [sum T M] FP32 copy (FP64 path screening)
  Real *fk;                           // [sum T K] base flows on outaged branches
  float *fk32;                        // [sum T K]
  Real *pold;                         // [sum T G] dispatch snapshot for the fused Adam ramp terms
  Real *uold;                         // [sum T G] on-status snapshot for the startup / shutdown terms
  Real *dP, *dQ;                      // [sum T n]
  Real *dZ;                           // [sum T Z]
  Real *pm, *pq, *pk;                 // contingency partials
  unsigned char *pmf;                 // row-partial flags (pm, pq are written and read only where set)
  int score;                          // 1: record per-(period, outage) scores (contingency screening)
  Real *pz;                           // score partials [n_mg][T][K] per instance (at pk0)
  Real *zs;                           // scores [sum T K] (at tk0)
  Real *gF;                           // [sum T M] dz/df
  Dc *gip;                            // adjoint DC products [sum T (Gb + 1)]
  Real *avf, *avo, *ad;               // branch-end adjoints [sum T M]
  Real *atx;                          // dPhi/dtau of the AC terms per transformer [sum T X]
  Dc *objp;                           // [n_obj_slots][N_TERMS] per-block objective terms: the
                                      // stage-1/2 blocks' slots, instance-major, then one per stage-5
                                      // device block, then one per stage-3 fold block
  int n_obj_slots, n_obj12;           // all slots; stage-1/2 slots
  int n_gen_slots;                    // stage-5 device-block slots (the fold slots follow them)
  long long n_pairs;                  // sum over instances of T G ((period, device) pairs)
  const int *slot_map;                // [n_obj12] stage-1/2 block (launch order) -> slot
  double *obj, *terms;                // [n_inst], [n_inst][N_TERMS]
  Real *g;                            // gradient [n_x]
  unsigned int *ticket;               // last-block counter of the stand-alone Adam kernel
  long long *step;                    // Adam step counter (written by closing kernels and that kernel)
  int step_off;                       // iteration k of a graph of several: it reads step + k
  // fused Adam (qg_solve): moments and hyper-parameters
  Real *am, *av;
  double lr, b1, b2, aeps;
  int paper_eps;
  const double *sched;                // optional per-iteration (lr, eps, beta) of a scheduled solve, [sched_len][3]
  int sched_len;
  double *trace;                      // optional objective trace (qg_solve), [trace_len][n_inst]
  long long *trace_step0;             // step count at the start of the traced solve
  int trace_len;
};

struct Plan {
  Spans s1, s2, s3, s4, s5;
  InstTab tab;
  long long n_x;
  int maxT;
  int maxTB;  // largest period chunk of a contingency block (sizes its shared memory)
  int ctg_bound;  // stage 2 runs its bound test (eager or on-demand path; the same for every instance)
  int ctg_lazy;   // stage 2 takes the on-demand path (k_ctg_margin runs before it)
  int n_gen_slots;  // objective reduction slots of the stage-5 device blocks
  int n_fold_slots; // objective reduction slots of the stage-3 fold blocks
  // sparse DC mode (instance 0 only): grids of the solve kernels
  int sp;
  int sp_inj_blocks;   // right-hand-side blocks of k_sp_inj (T more compute the mean injection)
  int sp_fw_blocks;    // k_sp_fwd rows / 8
  int sp_tail_blocks;  // k_sp_tail, 0 without a tail
  int sp_tail_ks;      // column splits of the dense tail product
  int sp_tail_kc;      // columns per split (a multiple of SP_BK)
  int sp_bw_blocks;    // k_sp_back forward pass
  int sp_bwa_blocks;   // k_sp_back adjoint pass
};

// Index-checked build (compiled with QG_CHECK_BOUNDS): the device keeps the address ranges of the
// library's device arrays (and of the caller's arrays a handle stores), and every access
// d.<array>[i] in the stage kernels is checked against them; a miss records the first bad source line
// and address and reads or writes a dummy word instead.  In the normal build these are no-ops.
void bounds_register(const void *p, size_t bytes);
void bounds_unregister(const void *p);
// 1: a checked access missed (line, address of the first); 0: none; -1: not an index-checked build.
int bounds_report(long long *line, unsigned long long *addr);

// One evaluation (with adam, the fused projected Adam update); with close, ended by the closing
// kernel (the objective sum; step += 1 with adam), else the objective is left in the slots for a
// later launch_finish.
template <typename Real, typename Dc>
cudaError_t launch_eval(const Dev<Real, Dc> &d, const Plan &P, const void *x, bool adam, bool close,
                        cudaStream_t s, cudaEvent_t *ev);

template <typename Real, typename Dc>
cudaError_t prepare_eval(int maxTB, bool score, bool lazy);

// Row maxima of instance I's line-outage block for the stage-2 bound test (Dev::lmax at I.lm0), from
// the block as stored (lodf, of type dtype); rerun whenever the block changes.
cudaError_t launch_lmax(const void *lodf, int dtype, float *lmax, const Inst &I, cudaStream_t s);

// Closing kernel of a graph of n fused iterations whose evaluations were launched without one: the
// last iteration's objective, then step += n.
template <typename Real, typename Dc>
cudaError_t launch_finish(const Dev<Real, Dc> &d, const Plan &P, int n, cudaStream_t s);

template <typename Real, typename Dc>
cudaError_t launch_round_project(const Dev<Real, Dc> &d, const Inst &I, const Real *x, const unsigned char *fixed,
                                 double *dist, Real *proj, cudaStream_t s);

template <typename Real, typename Dc>
cudaError_t launch_round_fix(const Dev<Real, Dc> &d, const Inst &I, Real *x, Real *lo, Real *hi, const int *idx,
                             int n, unsigned char *fixed, const Real *proj, cudaStream_t s);

template <typename Real>
cudaError_t launch_adam(Real *x, Real *m, Real *v, const Real *g, const Real *lo, const Real *hi, long long n,
                        long long *step, unsigned int *ticket, double lr, double b1, double b2, double eps,
                        int paper_eps, cudaStream_t s);

// Timed phases: the five stage kernels and the stand-alone Adam step.
constexpr int N_PHASES = 6;

}  // namespace qg
