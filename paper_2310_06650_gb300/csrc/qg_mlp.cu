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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qg.h"

namespace {

thread_local std::string g_mlp_error;

constexpr int BM = 64, BN = 64, BK = 32;  // GEMM block tile
constexpr int GEMM_THREADS = 128;         // 4 warps as 2 x 2, each 32 x 32

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Partial C[s][m][n] = sum over k in split s of A(m, k) B(k, n), where A(m, k) = A[m sam + k sak]
// and B(k, n) = B[k sbk + n sbn] (BF16, any strides), with warp-level BF16 MMA (m16n8k16, FP32
// accumulate).  Grid: (ceil(N/64), ceil(M/64), splits); each split covers kchunk of K.
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm(const __nv_bfloat16 *__restrict__ A, long long sam, long long sak,
                                                       const __nv_bfloat16 *__restrict__ B, long long sbk, long long sbn,
                                                       float *__restrict__ C, int M, int N, int K, int kchunk) {
  __shared__ __nv_bfloat16 sA[BM][BK + 8];
  __shared__ __nv_bfloat16 sB[BN][BK + 8];  // stored [n][k]
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int wm = wid >> 1, wn = wid & 1;
  const int g = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = kb; k0 < ke; k0 += BK) {
    // stage tiles; walk along whichever index is contiguous in memory
    for (int e = tid; e < BM * BK; e += GEMM_THREADS) {
      int r, c;
      if (sak == 1) { r = e / BK; c = e % BK; } else { c = e / BM; r = e % BM; }
      const int m = m0 + r, k = k0 + c;
      sA[r][c] = (m < M && k < ke) ? A[(long long)m * sam + (long long)k * sak] : zero;
    }
    for (int e = tid; e < BN * BK; e += GEMM_THREADS) {
      int r, c;
      if (sbk == 1) { r = e / BK; c = e % BK; } else { c = e / BN; r = e % BN; }
      const int n = n0 + r, k = k0 + c;
      sB[r][c] = (n < N && k < ke) ? B[(long long)k * sbk + (long long)n * sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + g, c = kk + 2 * tq;
        af[i][0] = pack2(sA[r][c], sA[r][c + 1]);
        af[i][1] = pack2(sA[r + 8][c], sA[r + 8][c + 1]);
        af[i][2] = pack2(sA[r][c + 8], sA[r][c + 9]);
        af[i][3] = pack2(sA[r + 8][c + 8], sA[r + 8][c + 9]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = wn * 32 + j * 8 + g, c = kk + 2 * tq;
        bf[j][0] = pack2(sB[r][c], sB[r][c + 1]);
        bf[j][1] = pack2(sB[r][c + 8], sB[r][c + 9]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
    }
    __syncthreads();
  }
  float *Cs = C + (long long)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + wm * 32 + i * 16 + g, c = n0 + wn * 32 + j * 8 + 2 * tq;
      if (r < M && c < N) Cs[(long long)r * N + c] = acc[i][j][0];
      if (r < M && c + 1 < N) Cs[(long long)r * N + c + 1] = acc[i][j][1];
      if (r + 8 < M && c < N) Cs[(long long)(r + 8) * N + c] = acc[i][j][2];
      if (r + 8 < M && c + 1 < N) Cs[(long long)(r + 8) * N + c + 1] = acc[i][j][3];
    }
}

// Epilogue of the forward layers: Z = sum of split-K partials + bias; optionally ReLU; writes Z
// (FP32) and the BF16 copy of the activation for the next GEMM.
__global__ void k_fwd_epi(const float *__restrict__ P, int splits, const float *__restrict__ bias, float *__restrict__ Z,
                          __nv_bfloat16 *__restrict__ Hb, int M, int N, int relu) {
  const long long total = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    float z = 0.f;
    for (int s = 0; s < splits; ++s) z += P[s * total + i];
    z += bias[i % N];
    Z[i] = z;
    if (Hb) Hb[i] = __float2bfloat16_rn(relu ? fmaxf(z, 0.f) : z);
  }
}

// Backward epilogue: D = sum of split-K partials, masked by relu'(Zmask) when given; FP32 and BF16 copies.
__global__ void k_bwd_epi(const float *__restrict__ P, int splits, const float *__restrict__ Zmask, float *__restrict__ D,
                          __nv_bfloat16 *__restrict__ Db, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int s = 0; s < splits; ++s) v += P[s * total + i];
    if (Zmask && !(Zmask[i] > 0.f)) v = 0.f;
    if (D) D[i] = v;
    if (Db) Db[i] = __float2bfloat16_rn(v);
  }
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// dY = 2 (Y - target) / (B * N) (BF16 for the backward GEMMs) and per-block partial sums of the
// squared error (FP64, fixed order).
__global__ void __launch_bounds__(256) k_loss(const float *__restrict__ Y, const float *__restrict__ Tg,
                                              __nv_bfloat16 *__restrict__ dYb, float *__restrict__ dY, double *part,
                                              long long total) {
  __shared__ double red[8];
  double acc = 0.0;
  const float sc = 2.0f / (float)total;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float r = Y[i] - Tg[i];
    acc += (double)r * (double)r;
    dY[i] = sc * r;
    dYb[i] = __float2bfloat16_rn(sc * r);
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

__global__ void k_loss_final(const double *part, int n, long long total, double *loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *loss = s / (double)total;
  }
}

// Bias gradient: column sums of D (B x N) in row order.
__global__ void k_colsum(const float *__restrict__ D, int B, int N, float *__restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int r = 0; r < B; ++r) s += D[(long long)r * N + c];
  out[c] = s;
}

// Adam on the FP32 master parameters; the BF16 weight copies follow.
__global__ void k_mlp_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                           long long n, float lr, float b1, float b2, float c1, float c2, float eps) {
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

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8)); }

}  // namespace

struct qg_mlp {
  int n_in, n_h, n_out, max_b;
  long long n_par;
  long long o_w1, o_b1, o_w2, o_b2, o_w3, o_b3;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  float *w = nullptr, *gw = nullptr, *am = nullptr, *av = nullptr;
  __nv_bfloat16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr;
  __nv_bfloat16 *xb = nullptr, *h1b = nullptr, *h2b = nullptr, *dyb = nullptr, *dz2b = nullptr, *dz1b = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dy = nullptr, *dz2 = nullptr, *dz1 = nullptr, *part = nullptr;
  double *lpart = nullptr;
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

// C (M x N, FP32 split-K partials in m->part) = A B; returns the number of splits used.
int gemm(qg_mlp *mm, const __nv_bfloat16 *A, long long sam, long long sak, const __nv_bfloat16 *B, long long sbk,
         long long sbn, int M, int N, int K) {
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int splits = std::max(1, std::min(64, (152 * 2 + tiles - 1) / tiles));
  splits = std::min(splits, std::max(1, K / 256));
  while ((long long)splits * M * N > mm->part_elems && splits > 1) --splits;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
  k_gemm<<<grid, GEMM_THREADS, 0, mm->stream>>>(A, sam, sak, B, sbk, sbn, mm->part, M, N, K, kchunk);
  return splits;
}

void forward(qg_mlp *m, int B) {
  const int H = m->n_h, I = m->n_in, O = m->n_out;
  int s = gemm(m, m->xb, I, 1, m->w1b, 1, I, B, H, I);
  k_fwd_epi<<<grid_for((long long)B * H), 256, 0, m->stream>>>(m->part, s, m->w + m->o_b1, m->z1, m->h1b, B, H, 1);
  s = gemm(m, m->h1b, H, 1, m->w2b, 1, H, B, H, H);
  k_fwd_epi<<<grid_for((long long)B * H), 256, 0, m->stream>>>(m->part, s, m->w + m->o_b2, m->z2, m->h2b, B, H, 1);
  s = gemm(m, m->h2b, H, 1, m->w3b, 1, H, B, O, H);
  k_fwd_epi<<<grid_for((long long)B * O), 256, 0, m->stream>>>(m->part, s, m->w + m->o_b3, m->y, nullptr, B, O, 0);
}

void refresh_bf16(qg_mlp *m) {
  const long long n1 = (long long)m->n_h * m->n_in, n2 = (long long)m->n_h * m->n_h, n3 = (long long)m->n_out * m->n_h;
  k_to_bf16<<<grid_for(n1), 256, 0, m->stream>>>(m->w + m->o_w1, m->w1b, n1);
  k_to_bf16<<<grid_for(n2), 256, 0, m->stream>>>(m->w + m->o_w2, m->w2b, n2);
  k_to_bf16<<<grid_for(n3), 256, 0, m->stream>>>(m->w + m->o_w3, m->w3b, n3);
}

}  // namespace

extern "C" {

int qg_mlp_create(qg_mlp **out, int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch, uint64_t seed) {
  g_mlp_error.clear();
  if (!out) return mfail(nullptr, QG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1) return mfail(nullptr, QG_ERR_INVALID_ARG, "sizes");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) return mfail(nullptr, QG_ERR_NO_DEVICE, "no CUDA device");
  qg_mlp *m = new qg_mlp();
  m->n_in = n_in; m->n_h = n_hidden; m->n_out = n_out; m->max_b = max_batch;
  m->o_w1 = 0; m->o_b1 = m->o_w1 + (long long)n_hidden * n_in;
  m->o_w2 = m->o_b1 + n_hidden; m->o_b2 = m->o_w2 + (long long)n_hidden * n_hidden;
  m->o_w3 = m->o_b2 + n_hidden; m->o_b3 = m->o_w3 + (long long)n_out * n_hidden;
  m->n_par = m->o_b3 + n_out;
  const long long B = max_batch, H = n_hidden, I = n_in, O = n_out;
  m->part_elems = std::max({64 * B * H, 64 * B * O, 8 * H * I, 8 * O * H, 8 * H * H, 8 * B * I});
  int rc = 0;
  if ((rc = mal(m, &m->w, m->n_par)) || (rc = mal(m, &m->gw, m->n_par)) || (rc = mal(m, &m->am, m->n_par)) ||
      (rc = mal(m, &m->av, m->n_par)) || (rc = mal(m, &m->w1b, H * I)) || (rc = mal(m, &m->w2b, H * H)) ||
      (rc = mal(m, &m->w3b, O * H)) || (rc = mal(m, &m->xb, B * I)) || (rc = mal(m, &m->h1b, B * H)) ||
      (rc = mal(m, &m->h2b, B * H)) || (rc = mal(m, &m->dyb, B * O)) || (rc = mal(m, &m->dz2b, B * H)) ||
      (rc = mal(m, &m->dz1b, B * H)) || (rc = mal(m, &m->z1, B * H)) || (rc = mal(m, &m->z2, B * H)) ||
      (rc = mal(m, &m->y, B * O)) || (rc = mal(m, &m->dy, B * O)) || (rc = mal(m, &m->dz2, B * H)) ||
      (rc = mal(m, &m->dz1, B * H)) || (rc = mal(m, &m->part, m->part_elems)) || (rc = mal(m, &m->lpart, 152 * 8))) {
    qg_mlp_destroy(m);
    return rc;
  }
  cudaMemset(m->gw, 0, m->n_par * sizeof(float));
  cudaMemset(m->am, 0, m->n_par * sizeof(float));
  cudaMemset(m->av, 0, m->n_par * sizeof(float));
  cudaMemset(m->w, 0, m->n_par * sizeof(float));
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
  const long long nx = (long long)batch * m->n_in;
  k_to_bf16<<<grid_for(nx), 256, 0, m->stream>>>(x, m->xb, nx);
  forward(m, batch);
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
  k_to_bf16<<<grid_for((long long)B * I), 256, 0, s>>>(x, m->xb, (long long)B * I);
  forward(m, B);
  const long long ny = (long long)B * O;
  const int lb = grid_for(ny);
  k_loss<<<lb, 256, 0, s>>>(m->y, target, m->dyb, m->dy, m->lpart, ny);
  if (loss) k_loss_final<<<1, 32, 0, s>>>(m->lpart, lb, ny, loss);
  // layer 3: dW3 = dY^T H2, db3 = colsum(dY), dH2 = dY W3 masked by relu'(Z2)
  int sp = gemm(m, m->dyb, 1, O, m->h2b, H, 1, O, H, B);
  k_bwd_epi<<<grid_for((long long)O * H), 256, 0, s>>>(m->part, sp, nullptr, m->gw + m->o_w3, nullptr, (long long)O * H);
  k_colsum<<<(O + 255) / 256, 256, 0, s>>>(m->dy, B, O, m->gw + m->o_b3);
  sp = gemm(m, m->dyb, O, 1, m->w3b, H, 1, B, H, O);
  k_bwd_epi<<<grid_for((long long)B * H), 256, 0, s>>>(m->part, sp, m->z2, m->dz2, m->dz2b, (long long)B * H);
  // layer 2
  sp = gemm(m, m->dz2b, 1, H, m->h1b, H, 1, H, H, B);
  k_bwd_epi<<<grid_for((long long)H * H), 256, 0, s>>>(m->part, sp, nullptr, m->gw + m->o_w2, nullptr, (long long)H * H);
  k_colsum<<<(H + 255) / 256, 256, 0, s>>>(m->dz2, B, H, m->gw + m->o_b2);
  sp = gemm(m, m->dz2b, H, 1, m->w2b, H, 1, B, H, H);
  k_bwd_epi<<<grid_for((long long)B * H), 256, 0, s>>>(m->part, sp, m->z1, m->dz1, m->dz1b, (long long)B * H);
  // layer 1
  sp = gemm(m, m->dz1b, 1, H, m->xb, I, 1, H, I, B);
  k_bwd_epi<<<grid_for((long long)H * I), 256, 0, s>>>(m->part, sp, nullptr, m->gw + m->o_w1, nullptr, (long long)H * I);
  k_colsum<<<(H + 255) / 256, 256, 0, s>>>(m->dz1, B, H, m->gw + m->o_b1);
  // Adam
  if (lr > 0) {
    m->step += 1;
    const double c1 = 1.0 / (1.0 - std::pow(beta1, (double)m->step));
    const double c2 = 1.0 / (1.0 - std::pow(beta2, (double)m->step));
    k_mlp_adam<<<grid_for(m->n_par), 256, 0, s>>>(m->w, m->gw, m->am, m->av, m->n_par, (float)lr, (float)beta1,
                                                  (float)beta2, (float)c1, (float)c2, 1e-8f);
    refresh_bf16(m);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QG_OK : mfail(m, QG_ERR_CUDA, cudaGetErrorString(e));
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
