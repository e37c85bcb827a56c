// Learned warm start: a three-layer MLP (BF16 weights and activations into FP32-accumulating
// tensor-core GEMMs) that maps a load profile to an initial dispatch, voltage magnitudes and
// angles; trained on the GPU by its own forward / backward kernels and an Adam step.
//
//   Z1 = X W1^T + b1,  H1 = relu(Z1),  Z2 = H1 W2^T + b2,  H2 = relu(Z2),  Y = H2 W3^T + b3,
//   loss = mean((Y - target)^2).
// GEMM operands are rounded to BF16 where they enter a GEMM (X, H1, H2, the weights, and the
// back-propagated dY, dZ2, dZ1); accumulation is FP32; master weights, biases, moments and the
// loss are FP32 / FP64.  Every reduction has a fixed order (split-K partials are summed in a
// second pass), so results are bitwise repeatable.
//
// The GEMMs run on the fifth-generation tensor cores: C[m][n] = sum_k A[m][k] B[n][k] with both
// operands BF16 and K-contiguous, staged by TMA (128-byte swizzle) through a ring of shared-memory
// stages, multiplied by tcgen05.mma (M = 128) issued from one thread into a TMEM accumulator, and
// read back with tcgen05.ld for the FP32 partial-sum epilogue.  Every product of the network is
// put in that form: the layers run with the weights as A (their rows fill the 128 TMEM lanes) and
// the batch as B (N = 64), writing the transposed tile; the weight gradients take transposed BF16
// copies of the activations and back-propagated terms (batch-contiguous), the input gradients
// transposed BF16 copies of W2 and W3.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qg.h"

namespace {

thread_local std::string g_mlp_error;

constexpr int UM = 128;              // tile rows: the MMA's M, one TMEM lane each
constexpr int UK = 64;               // K per stage: 64 BF16 = one 128-byte swizzle span per row
constexpr int UTHREADS = 128;        // warp 0: TMA producer, warp 1: MMA issuer, warp 2: TMEM owner; all: epilogue
constexpr unsigned long long WAIT_NS = 1000000000ull;  // a wait gives up after 1 s (error flag, clean exit)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the completion of the barrier's phase `parity`.  Gives up after WAIT_NS (or 2^30 polls),
// or at once when another thread of the block has given up (abort != 0 and honour_abort); returns
// whether the phase completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort, bool honour_abort) {
  const unsigned long long t0 = gtime();
  for (unsigned it = 0; it < (1u << 30); ++it) {
    if (mbar_test(b, parity)) return true;
    if (honour_abort && *abort) return false;
    if (gtime() - t0 > WAIT_NS) break;
  }
  *abort = 1;
  return false;
}

// TMA: the box at (c0 = K offset in elements, c1 = row) of a 2-D BF16 tensor map into shared memory,
// completing `bytes` on the barrier.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the 128-byte swizzle: rows
// of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1, layout
// SWIZZLE_128B; the leading byte offset is unused for this layout.  The tile starts on a 1024-byte
// boundary, so the K step inside a row is a plain start-address offset (32 bytes per 16 elements).
__device__ __forceinline__ uint64_t umma_desc(const void *tile) {
  const uint32_t a = smem_u32(tile);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t umma_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the barrier completes once every tcgen05.mma this thread issued before has completed
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// programmatic dependent launch: wait for the preceding kernels' results (a no-op without it)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN, int STAGES>
constexpr size_t umma_smem_bytes() {
  return (size_t)STAGES * (UM * UK * 2 + BN * UK * 2) + 1024;  // + alignment of the first tile to 1024 bytes
}

// Partial C[s] of split s (FP32, M x N row-major, or its transpose N x M when trans) =
//   sum over the K blocks [s kbps, (s + 1) kbps) of A[m][k] B[n][k],
// A (M x K) and B (N x K) BF16 behind the tensor maps tA (box 64 x 128) and tB (box 64 x BN); rows
// and K beyond the tensors read as zeros.  Grid (ceil(M/128), ceil(N/BN), splits), 128 threads.
// Launched as a programmatic dependent of the previous kernel: with a_static (A is not written by
// the two kernels before it: the weights) the first stages' A tiles are requested before the wait.
// A wait that runs out sets *err, drains what this block started and returns.
template <int BN, int STAGES>
__global__ void __launch_bounds__(UTHREADS, 1)
    k_umma_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, float *__restrict__ P,
                int M, int N, int nkb, int kbps, int trans, int a_static, int *err) {
  constexpr uint32_t A_BYTES = UM * UK * 2, B_BYTES = BN * UK * 2;
  constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;  // a power of two >= 32
  static_assert((BN & (BN - 1)) == 0 && BN >= 16 && BN <= 256, "BN");
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *sA = base, *sB = base + STAGES * A_BYTES;
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accf;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort, s_issued, s_consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * UM, n0 = blockIdx.y * BN;
  const int kb0 = blockIdx.z * kbps, nk = min(kbps, nkb - kb0);  // >= 1: the host sizes the splits so
  volatile int *abort = &s_abort;
  const int pre = a_static ? min(nk, STAGES) : 0;  // stages whose A tile is requested before the wait
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accf, 1);
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int kb = 0; kb < pre; ++kb) {
      mbar_expect_tx(&full[kb], A_BYTES + B_BYTES);
      tma_load_2d(sA + kb * A_BYTES, &tA, &full[kb], (kb0 + kb) * UK, m0);
    }
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  pdl_wait();  // B, and the partial buffer this kernel overwrites, belong to the kernels before it
  if (warp == 0 && lane == 0) {  // producer: stage s holds K block kb, its u-th use
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t u = (uint32_t)(kb / STAGES);
      const int kx = (kb0 + kb) * UK;  // a multiple of 64 elements: 128-byte aligned
      if (kb >= pre) {
        if (kb >= STAGES && !mbar_wait(&empty[s], (u - 1) & 1, abort, true)) break;
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        tma_load_2d(sA + s * A_BYTES, &tA, &full[s], kx, m0);
      }
      tma_load_2d(sB + s * B_BYTES, &tB, &full[s], kx, n0);
      issued = kb + 1;
    }
    s_issued = max(issued, pre);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    constexpr uint32_t IDESC = umma_idesc<BN>();
    int consumed = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)(kb / STAGES) & 1, abort, true)) break;
      tc_fence_after();
      const uint64_t ad = umma_desc(sA + s * A_BYTES), bd = umma_desc(sB + s * B_BYTES);
#pragma unroll
      for (int j = 0; j < UK / 16; ++j)  // K = 16 per MMA: 32 bytes (2 descriptor units) along the row
        umma_bf16(tmem, ad + 2 * j, bd + 2 * j, IDESC, (kb | j) != 0);
      umma_commit(&empty[s]);  // stage s is free once these MMAs have read it
      consumed = kb + 1;
    }
    s_consumed = consumed;
    umma_commit(&accf);  // every MMA above has completed (also after an abort)
  }
  __syncwarp();
  // the accumulator is complete (or, after an abort, no MMA is in flight any more); the flag is read
  // after a barrier so that every warp takes the same branch into the warp-collective TMEM loads
  mbar_wait(&accf, 0, abort, false);
  tc_fence_after();
  __syncthreads();
  if (!*abort) {
    const int m = m0 + warp * 32 + lane;
    float *Ps = P + (long long)blockIdx.z * M * N;
    if (trans) {  // C^T: for each column the warp's 32 lanes (rows) write 32 consecutive floats
#pragma unroll 1
      for (int c0 = 0; c0 < BN && n0 + c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (m < M)
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (n0 + c0 + i < N) Ps[(long long)(n0 + c0 + i) * M + m] = v[i];
      }
    } else {  // C: 32 x 32 pieces turned around in shared memory, each row written by the warp's lanes;
      // the stage buffers are free by now (every TMA copy was consumed, every MMA has completed)
      static_assert(4 * 32 * 33 * sizeof(float) <= STAGES * (A_BYTES + B_BYTES), "epilogue tile");
      float(*t)[33] = reinterpret_cast<float(*)[33]>(base) + warp * 32;
#pragma unroll 1
      for (int c0 = 0; c0 < BN && n0 + c0 < N; c0 += 32) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) t[lane][i] = v[i];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c0 + 16), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) t[lane][16 + i] = v[i];
        __syncwarp();
        const int n = n0 + c0 + lane;
        for (int r = 0; r < 32; ++r) {
          const int mr = m0 + warp * 32 + r;
          if (mr < M && n < N) Ps[(long long)mr * N + n] = t[r][lane];
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort) {
    atomicExch(err, 1);
    // copies still in flight land in this block's shared memory: wait for them (bounded) before exit
    for (int kb = s_consumed; kb < s_issued; ++kb) mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1, abort, false);
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Transposed BF16 copy: dst[c][r] (row stride ldd) = src[r][c] (FP32, rows x cols, row stride lds),
// through a 32 x 33 shared tile so that both sides are coalesced.  Grid (ceil(cols/32), ceil(rows/32)),
// block (32, 8).
__global__ void k_transpose_bf16(const float *__restrict__ src, long long lds, __nv_bfloat16 *__restrict__ dst,
                                 long long ldd, int rows, int cols) {
  pdl_wait();
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < rows && c < cols) ? src[(long long)r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[(long long)c * ldd + r] = __float2bfloat16_rn(t[threadIdx.x][i]);
  }
}

// BF16 copy with a padded row stride: dst[r][c] (stride ldd) = src[r][c] (FP32, stride lds).
// Grid (column chunks of 256, rows; the rows strided by gridDim.y): no index division per element.
__global__ void k_rows_bf16(const float *__restrict__ src, long long lds, __nv_bfloat16 *__restrict__ dst, long long ldd,
                            int rows, int cols) {
  pdl_wait();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) dst[(long long)r * ldd + c] = __float2bfloat16_rn(src[(long long)r * lds + c]);
}

// Epilogue of the forward layers: Z = sum of split-K partials + bias (M x N); optionally ReLU;
// writes Z (FP32) and the activation in BF16 for the next GEMMs: row-major with row stride ldh
// (Hb) and transposed with row stride ldt (HbT, batch-contiguous).
__global__ void k_fwd_epi(const float *__restrict__ P, int splits, const float *__restrict__ bias, float *__restrict__ Z,
                          __nv_bfloat16 *__restrict__ Hb, long long ldh, __nv_bfloat16 *__restrict__ HbT, long long ldt,
                          int M, int N, int relu) {
  pdl_wait();
  const long long total = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    float z = 0.f;
    for (int s = 0; s < splits; ++s) z += P[s * total + i];
    const long long r = i / N, c = i - r * N;
    z += bias[c];
    Z[i] = z;
    const __nv_bfloat16 h = __float2bfloat16_rn(relu ? fmaxf(z, 0.f) : z);
    if (Hb) Hb[r * ldh + c] = h;
    if (HbT) HbT[c * ldt + r] = h;
  }
}

// Backward epilogue: D = sum of split-K partials (rows x cols), masked by relu'(Zmask) when given;
// FP32 (D, dense), BF16 row-major with row stride ldd (Db) and BF16 transposed with row stride
// ldt (DbT).
__global__ void k_bwd_epi(const float *__restrict__ P, int splits, const float *__restrict__ Zmask, float *__restrict__ D,
                          __nv_bfloat16 *__restrict__ Db, long long ldd, __nv_bfloat16 *__restrict__ DbT, long long ldt,
                          int rows, int cols) {
  pdl_wait();
  const long long total = (long long)rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int s = 0; s < splits; ++s) v += P[s * total + i];
    if (Zmask && !(Zmask[i] > 0.f)) v = 0.f;
    if (D) D[i] = v;
    if (Db || DbT) {
      const long long r = i / cols, c = i - r * cols;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      if (Db) Db[r * ldd + c] = h;
      if (DbT) DbT[c * ldt + r] = h;
    }
  }
}

// dY = 2 (Y - target) / (B * N) (BF16 for the backward GEMMs) and per-block partial sums of the
// squared error (FP64, fixed order).
__global__ void __launch_bounds__(256) k_loss(const float *__restrict__ Y, const float *__restrict__ Tg,
                                              __nv_bfloat16 *__restrict__ dYb, long long ldo,
                                              __nv_bfloat16 *__restrict__ dYbT, long long ldt, float *__restrict__ dY,
                                              double *part, int rows, int cols) {
  pdl_wait();
  __shared__ double red[8];
  double acc = 0.0;
  const long long total = (long long)rows * cols;
  const float sc = 2.0f / (float)total;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float r = Y[i] - Tg[i];
    acc += (double)r * (double)r;
    dY[i] = sc * r;
    const long long b = i / cols, o = i - b * cols;
    const __nv_bfloat16 h = __float2bfloat16_rn(sc * r);
    dYb[b * ldo + o] = h;
    dYbT[o * ldt + b] = h;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// The mean of the block partials: one block of 256 threads, strided sums then a shuffle and
// shared-memory tree (a fixed order).
__global__ void __launch_bounds__(256) k_loss_final(const double *part, int n, long long total, double *loss) {
  pdl_wait();
  __shared__ double red[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *loss = t / (double)total;
  }
}

// Bias gradient: column sums of D (B x N) in row order.
__global__ void k_colsum(const float *__restrict__ D, int B, int N, float *__restrict__ out) {
  pdl_wait();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int r = 0; r < B; ++r) s += D[(long long)r * N + c];
  out[c] = s;
}

// Adam on the FP32 master parameters; the BF16 weight copies follow.
__global__ void k_mlp_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                           long long n, float lr, float b1, float b2, float c1, float c2, float eps) {
  pdl_wait();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// Deterministic counter-based normal draws (Box-Muller on a splitmix64 stream) for the initial weights.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_init(float *__restrict__ w, long long n, float scale, uint64_t seed, long long offset) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ (uint64_t)(offset + i) * 2ull);
    const uint64_t b = splitmix64(seed ^ ((uint64_t)(offset + i) * 2ull + 1ull));
    const float u1 = ((a >> 40) + 1.0f) * (1.0f / 16777217.0f);
    const float u2 = (b >> 40) * (1.0f / 16777216.0f);
    w[i] = scale * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
  }
}

// Launch as a programmatic dependent of the previous kernel in the stream (each kernel waits with
// griddepcontrol.wait before it touches what earlier kernels wrote or read).
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8)); }

long long pad8(long long n) { return (n + 7) / 8 * 8; }  // BF16 row strides: multiples of 16 bytes (TMA)

}  // namespace

struct qg_mlp {
  int n_in, n_h, n_out, max_b;
  long long ld_i, ld_h, ld_o, ld_b;  // padded BF16 row strides for rows of I, H, O and batch elements
  long long n_par;
  long long o_w1, o_b1, o_w2, o_b2, o_w3, o_b3;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  float *w = nullptr, *gw = nullptr, *am = nullptr, *av = nullptr;
  // BF16 GEMM operands, all K-contiguous: weights [H][ld_i], [H][ld_h], [O][ld_h] and the transposed
  // W2^T [H][ld_h], W3^T [H][ld_o]; activations row-major [B][ld_*] and transposed [features][ld_b]
  __nv_bfloat16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr, *w2t = nullptr, *w3t = nullptr;
  __nv_bfloat16 *xb = nullptr, *xt = nullptr, *h1b = nullptr, *h1t = nullptr, *h2b = nullptr, *h2t = nullptr;
  __nv_bfloat16 *dyb = nullptr, *dyt = nullptr, *dz2b = nullptr, *dz2t = nullptr, *dz1t = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dy = nullptr, *dz2 = nullptr, *dz1 = nullptr, *part = nullptr;
  double *lpart = nullptr;
  int *d_err = nullptr;  // set by a GEMM block whose pipeline wait ran out
  long long part_elems = 0;
  long long step = 0;
  std::string err;
};

namespace {

int mfail(qg_mlp *m, int code, const std::string &msg) {
  if (m) m->err = msg;
  g_mlp_error = msg;
  return code;
}

template <typename T>
int mal(qg_mlp *m, T **p, size_t n) {
  cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return mfail(m, QG_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  m->allocs.push_back(*p);
  return QG_OK;
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// 2-D tensor map of a BF16 matrix (rows x cols, row stride ld elements, a multiple of 8) with a box
// of 64 columns (128 bytes, the swizzle span) x box_rows rows; reads outside the matrix give zeros.
int make_map(qg_mlp *m, CUtensorMap *map, const __nv_bfloat16 *ptr, long long rows, long long cols, long long ld,
             int box_rows) {
  const auto enc = tensor_map_encoder();
  if (!enc) return mfail(m, QG_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)UK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return mfail(m, QG_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return QG_OK;
}

template <int BN, int STAGES>
cudaError_t umma_prepare() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(k_umma_gemm<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)umma_smem_bytes<BN, STAGES>());
  });
  return e;
}

// Split-K partials of C = A B^T (A: M x K with row stride lda, B: N x K with row stride ldb, both BF16)
// into mm->part: [splits][M][N], or [splits][N][M] with trans; with dst, C itself (one split) into dst.  Returns the number of splits, or 0
// after recording an error.  Narrow products (N <= 64: the batch) take 64-column tiles and a
// 4-stage ring; wide ones (the weight gradients, K = the batch) 256-column tiles and 2 stages.
// a_static: A is a weight copy (not written by the kernels just before), requested before the wait.
int gemm(qg_mlp *mm, const __nv_bfloat16 *A, long long lda, int M, const __nv_bfloat16 *B, long long ldb, int N, int K,
         bool trans, bool a_static, float *dst = nullptr) {
  const bool narrow = N <= 64;
  const int BN = narrow ? 64 : 256;
  const long long tiles = (long long)((M + UM - 1) / UM) * ((N + BN - 1) / BN);
  const int nkb = (K + UK - 1) / UK;
  int splits = dst ? 1 : (int)std::max(1LL, std::min<long long>({64LL, (long long)nkb, (2LL * 152 + tiles - 1) / tiles}));
  while (splits > 1 && (long long)splits * M * N > mm->part_elems) --splits;
  const int kbps = (nkb + splits - 1) / splits;
  splits = (nkb + kbps - 1) / kbps;  // every split has at least one K block
  CUtensorMap ta, tb;
  int rc = make_map(mm, &ta, A, M, K, lda, UM);
  if (!rc) rc = make_map(mm, &tb, B, N, K, ldb, BN);
  if (rc) return 0;
  const dim3 grid((M + UM - 1) / UM, (N + BN - 1) / BN, splits);
  float *out = dst ? dst : mm->part;
  cudaError_t e;
  if (narrow) {
    e = umma_prepare<64, 4>();
    if (e == cudaSuccess)
      e = pdl_launch(k_umma_gemm<64, 4>, grid, dim3(UTHREADS), umma_smem_bytes<64, 4>(), mm->stream, ta, tb, out, M,
                     N, nkb, kbps, trans ? 1 : 0, a_static ? 1 : 0, mm->d_err);
  } else {
    e = umma_prepare<256, 2>();
    if (e == cudaSuccess)
      e = pdl_launch(k_umma_gemm<256, 2>, grid, dim3(UTHREADS), umma_smem_bytes<256, 2>(), mm->stream, ta, tb, out,
                     M, N, nkb, kbps, trans ? 1 : 0, a_static ? 1 : 0, mm->d_err);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    mfail(mm, QG_ERR_CUDA, std::string("tensor-core GEMM launch: ") + cudaGetErrorString(e));
    return 0;
  }
  return splits;
}

// x (batch x I, FP32) into the BF16 operand xb [B][ld_i] and, for training (the first layer's weight
// gradient), xt [I][ld_b]
void load_x(qg_mlp *m, const float *x, int B, bool transposed) {
  pdl_launch(k_rows_bf16, dim3((m->n_in + 255) / 256, std::min(B, 65535)), dim3(256), 0, m->stream, x, m->n_in, m->xb,
             m->ld_i, B, m->n_in);
  if (transposed)
    pdl_launch(k_transpose_bf16, dim3((m->n_in + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, m->stream, x, m->n_in, m->xt,
               m->ld_b, B, m->n_in);
}

// Forward pass: the layers as C^T = W act^T (weights as the 128-row operand, the batch as N).
int forward(qg_mlp *m, int B) {
  const int H = m->n_h, I = m->n_in, O = m->n_out;
  int s = gemm(m, m->w1b, m->ld_i, H, m->xb, m->ld_i, B, I, true, true);
  if (!s) return QG_ERR_CUDA;
  pdl_launch(k_fwd_epi, dim3(grid_for((long long)B * H)), dim3(256), 0, m->stream, m->part, s, m->w + m->o_b1, m->z1,
             m->h1b, m->ld_h, m->h1t, m->ld_b, B, H, 1);
  if (!(s = gemm(m, m->w2b, m->ld_h, H, m->h1b, m->ld_h, B, H, true, true))) return QG_ERR_CUDA;
  pdl_launch(k_fwd_epi, dim3(grid_for((long long)B * H)), dim3(256), 0, m->stream, m->part, s, m->w + m->o_b2, m->z2,
             m->h2b, m->ld_h, m->h2t, m->ld_b, B, H, 1);
  if (!(s = gemm(m, m->w3b, m->ld_h, O, m->h2b, m->ld_h, B, H, true, true))) return QG_ERR_CUDA;
  pdl_launch(k_fwd_epi, dim3(grid_for((long long)B * O)), dim3(256), 0, m->stream, m->part, s, m->w + m->o_b3, m->y,
             nullptr, 0, nullptr, 0, B, O, 0);
  return QG_OK;
}

// BF16 operand copies of the FP32 master weights: W1, W2, W3 row-major (padded) and W2^T, W3^T.
void refresh_bf16(qg_mlp *m) {
  const int H = m->n_h, I = m->n_in, O = m->n_out;
  cudaStream_t s = m->stream;
  pdl_launch(k_rows_bf16, dim3((I + 255) / 256, std::min(H, 65535)), dim3(256), 0, s, m->w + m->o_w1, I, m->w1b, m->ld_i,
             H, I);
  pdl_launch(k_rows_bf16, dim3((H + 255) / 256, std::min(H, 65535)), dim3(256), 0, s, m->w + m->o_w2, H, m->w2b, m->ld_h,
             H, H);
  pdl_launch(k_rows_bf16, dim3((H + 255) / 256, std::min(O, 65535)), dim3(256), 0, s, m->w + m->o_w3, H, m->w3b, m->ld_h,
             O, H);
  pdl_launch(k_transpose_bf16, dim3((H + 31) / 32, (H + 31) / 32), dim3(32, 8), 0, s, m->w + m->o_w2, H, m->w2t,
             m->ld_h, H, H);
  pdl_launch(k_transpose_bf16, dim3((H + 31) / 32, (O + 31) / 32), dim3(32, 8), 0, s, m->w + m->o_w3, H, m->w3t,
             m->ld_o, O, H);
}

}  // namespace

extern "C" {

int qg_mlp_create(qg_mlp **out, int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch, uint64_t seed) {
  g_mlp_error.clear();
  if (!out) return mfail(nullptr, QG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1) return mfail(nullptr, QG_ERR_INVALID_ARG, "sizes");
  if (max_batch > 64) return mfail(nullptr, QG_ERR_UNSUPPORTED, "max_batch above 64 (one 64-column GEMM tile)");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) return mfail(nullptr, QG_ERR_NO_DEVICE, "no CUDA device");
  if (!tensor_map_encoder()) return mfail(nullptr, QG_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  qg_mlp *m = new qg_mlp();
  m->n_in = n_in; m->n_h = n_hidden; m->n_out = n_out; m->max_b = max_batch;
  m->ld_i = pad8(n_in); m->ld_h = pad8(n_hidden); m->ld_o = pad8(n_out); m->ld_b = pad8(max_batch);
  m->o_w1 = 0; m->o_b1 = m->o_w1 + (long long)n_hidden * n_in;
  m->o_w2 = m->o_b1 + n_hidden; m->o_b2 = m->o_w2 + (long long)n_hidden * n_hidden;
  m->o_w3 = m->o_b2 + n_hidden; m->o_b3 = m->o_w3 + (long long)n_out * n_hidden;
  m->n_par = m->o_b3 + n_out;
  const long long B = max_batch, H = n_hidden, I = n_in, O = n_out;
  const long long li = m->ld_i, lh = m->ld_h, lo = m->ld_o, lb = m->ld_b;
  m->part_elems = std::max({64 * B * H, 64 * B * O, H * I, O * H, H * H});
  int rc = 0;
  if ((rc = mal(m, &m->w, m->n_par)) || (rc = mal(m, &m->gw, m->n_par)) || (rc = mal(m, &m->am, m->n_par)) ||
      (rc = mal(m, &m->av, m->n_par)) || (rc = mal(m, &m->w1b, H * li)) || (rc = mal(m, &m->w2b, H * lh)) ||
      (rc = mal(m, &m->w3b, O * lh)) || (rc = mal(m, &m->w2t, H * lh)) || (rc = mal(m, &m->w3t, H * lo)) ||
      (rc = mal(m, &m->xb, B * li)) || (rc = mal(m, &m->xt, I * lb)) || (rc = mal(m, &m->h1b, B * lh)) ||
      (rc = mal(m, &m->h1t, H * lb)) || (rc = mal(m, &m->h2b, B * lh)) || (rc = mal(m, &m->h2t, H * lb)) ||
      (rc = mal(m, &m->dyb, B * lo)) || (rc = mal(m, &m->dyt, O * lb)) || (rc = mal(m, &m->dz2b, B * lh)) ||
      (rc = mal(m, &m->dz2t, H * lb)) || (rc = mal(m, &m->dz1t, H * lb)) || (rc = mal(m, &m->z1, B * H)) ||
      (rc = mal(m, &m->z2, B * H)) || (rc = mal(m, &m->y, B * O)) || (rc = mal(m, &m->dy, B * O)) ||
      (rc = mal(m, &m->dz2, B * H)) || (rc = mal(m, &m->dz1, B * H)) || (rc = mal(m, &m->part, m->part_elems)) ||
      (rc = mal(m, &m->lpart, 152 * 8)) || (rc = mal(m, &m->d_err, 1))) {
    qg_mlp_destroy(m);
    return rc;
  }
  cudaMemset(m->gw, 0, m->n_par * sizeof(float));
  cudaMemset(m->am, 0, m->n_par * sizeof(float));
  cudaMemset(m->av, 0, m->n_par * sizeof(float));
  cudaMemset(m->w, 0, m->n_par * sizeof(float));
  cudaMemset(m->d_err, 0, sizeof(int));
  // He initialisation for the ReLU layers, a smaller scale for the linear output layer; zero biases
  k_init<<<grid_for(H * I), 256>>>(m->w + m->o_w1, H * I, sqrtf(2.f / (float)I), seed, 0);
  k_init<<<grid_for(H * H), 256>>>(m->w + m->o_w2, H * H, sqrtf(2.f / (float)H), seed, H * I);
  k_init<<<grid_for(O * H), 256>>>(m->w + m->o_w3, O * H, sqrtf(1.f / (float)H), seed, H * I + H * H);
  refresh_bf16(m);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    mfail(m, QG_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e));
    qg_mlp_destroy(m);
    return QG_ERR_CUDA;
  }
  *out = m;
  return QG_OK;
}

void qg_mlp_destroy(qg_mlp *m) {
  if (!m) return;
  for (void *p : m->allocs) cudaFree(p);
  delete m;
}

int64_t qg_mlp_num_params(const qg_mlp *m) { return m ? m->n_par : 0; }

int qg_mlp_set_stream(qg_mlp *m, void *stream) {
  if (!m) return QG_ERR_INVALID_ARG;
  m->stream = (cudaStream_t)stream;
  return QG_OK;
}

int qg_mlp_forward(qg_mlp *m, const float *x, int32_t batch, float *y) {
  if (!m || !x || !y || batch < 1 || batch > m->max_b) return m ? mfail(m, QG_ERR_INVALID_ARG, "forward arguments") : QG_ERR_INVALID_ARG;
  load_x(m, x, batch, false);
  int rc = forward(m, batch);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(y, m->y, sizeof(float) * batch * m->n_out, cudaMemcpyDeviceToDevice, m->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? QG_OK : mfail(m, QG_ERR_CUDA, cudaGetErrorString(e));
}

int qg_mlp_train_step(qg_mlp *m, const float *x, const float *target, int32_t batch, double lr, double beta1,
                      double beta2, double *loss) {
  if (!m || !x || !target || batch < 1 || batch > m->max_b)
    return m ? mfail(m, QG_ERR_INVALID_ARG, "train arguments") : QG_ERR_INVALID_ARG;
  const int B = batch, H = m->n_h, I = m->n_in, O = m->n_out;
  cudaStream_t s = m->stream;
  load_x(m, x, B, true);
  int rc = forward(m, B);
  if (rc) return rc;
  const long long ny = (long long)B * O;
  const int lb = grid_for(ny);
  pdl_launch(k_loss, dim3(lb), dim3(256), 0, s, m->y, target, m->dyb, m->ld_o, m->dyt, m->ld_b, m->dy, m->lpart, B,
             O);
  if (loss) pdl_launch(k_loss_final, dim3(1), dim3(256), 0, s, m->lpart, lb, ny, loss);
  // layer 3: dW3 = dY^T H2 (K = the batch: one split, written straight into the gradient),
  // db3 = colsum(dY), dH2 = dY W3 masked by relu'(Z2)
  int sp = gemm(m, m->dyt, m->ld_b, O, m->h2t, m->ld_b, H, B, false, false, m->gw + m->o_w3);
  if (!sp) return QG_ERR_CUDA;
  pdl_launch(k_colsum, dim3((O + 255) / 256), dim3(256), 0, s, m->dy, B, O, m->gw + m->o_b3);
  if (!(sp = gemm(m, m->w3t, m->ld_o, H, m->dyb, m->ld_o, B, O, true, true))) return QG_ERR_CUDA;
  pdl_launch(k_bwd_epi, dim3(grid_for((long long)B * H)), dim3(256), 0, s, m->part, sp, m->z2, m->dz2, m->dz2b, m->ld_h,
             m->dz2t, m->ld_b, B, H);
  // layer 2
  if (!(sp = gemm(m, m->dz2t, m->ld_b, H, m->h1t, m->ld_b, H, B, false, false, m->gw + m->o_w2))) return QG_ERR_CUDA;
  pdl_launch(k_colsum, dim3((H + 255) / 256), dim3(256), 0, s, m->dz2, B, H, m->gw + m->o_b2);
  if (!(sp = gemm(m, m->w2t, m->ld_h, H, m->dz2b, m->ld_h, B, H, true, true))) return QG_ERR_CUDA;
  pdl_launch(k_bwd_epi, dim3(grid_for((long long)B * H)), dim3(256), 0, s, m->part, sp, m->z1, m->dz1, nullptr, 0,
             m->dz1t, m->ld_b, B, H);
  // layer 1
  if (!(sp = gemm(m, m->dz1t, m->ld_b, H, m->xt, m->ld_b, I, B, false, false, m->gw + m->o_w1))) return QG_ERR_CUDA;
  pdl_launch(k_colsum, dim3((H + 255) / 256), dim3(256), 0, s, m->dz1, B, H, m->gw + m->o_b1);
  // Adam
  if (lr > 0) {
    m->step += 1;
    const double c1 = 1.0 / (1.0 - std::pow(beta1, (double)m->step));
    const double c2 = 1.0 / (1.0 - std::pow(beta2, (double)m->step));
    pdl_launch(k_mlp_adam, dim3(grid_for(m->n_par)), dim3(256), 0, s, m->w, m->gw, m->am, m->av, m->n_par, (float)lr,
               (float)beta1, (float)beta2, (float)c1, (float)c2, 1e-8f);
    refresh_bf16(m);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QG_OK : mfail(m, QG_ERR_CUDA, cudaGetErrorString(e));
}

int qg_mlp_check(qg_mlp *m) {
  if (!m) return QG_ERR_INVALID_ARG;
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, QG_ERR_CUDA, cudaGetErrorString(e));
  if (flag) return mfail(m, QG_ERR_CUDA, "a tensor-core GEMM pipeline wait ran out (1 s); its results are invalid");
  return QG_OK;
}

int qg_mlp_get_params(qg_mlp *m, float *w) {
  if (!m || !w) return QG_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(w, m->w, sizeof(float) * m->n_par, cudaMemcpyDeviceToDevice, m->stream);
  return e == cudaSuccess ? QG_OK : mfail(m, QG_ERR_CUDA, cudaGetErrorString(e));
}

int qg_mlp_set_params(qg_mlp *m, const float *w) {
  if (!m || !w) return QG_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(m->w, w, sizeof(float) * m->n_par, cudaMemcpyDeviceToDevice, m->stream);
  if (e != cudaSuccess) return mfail(m, QG_ERR_CUDA, cudaGetErrorString(e));
  refresh_bf16(m);
  return QG_OK;
}

int qg_mlp_get_grads(qg_mlp *m, float *g) {
  if (!m || !g) return QG_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(g, m->gw, sizeof(float) * m->n_par, cudaMemcpyDeviceToDevice, m->stream);
  return e == cudaSuccess ? QG_OK : mfail(m, QG_ERR_CUDA, cudaGetErrorString(e));
}

const char *qg_mlp_last_error(const qg_mlp *m) { return m ? m->err.c_str() : g_mlp_error.c_str(); }

}  // extern "C"
