// rhd_surrogate.cuh -- the learned warm start: a small MLP that maps a cell's
// state to a guess of its updated gas temperature and group energies, trained
// on cells the solver itself has updated, and used as the starting point of
// the Newton iteration (which then runs to the same tolerance, and falls back
// to the cold start wherever the guess does not converge).
//
// Network: features (2 N_g + 4) -> 128 -> 128 -> 128 -> N_g + 1, GELU after
// the three hidden layers; BF16 weights and activations, FP32 accumulation on
// the tensor cores (rhd_tc.cuh), FP32 master parameters and Adam moments.
// Features of a cell (raw, before standardisation): ln rho, ln T,
// ln(E_g / a T^4) (N_g), |F_g| / (c E_g) (N_g), |v| / c, ln(c rho kappa0 dt).
// Targets: ln(T_new / T), ln(E_g,new / E_g) (N_g).  Features and targets are
// standardised with per-column means and deviations fitted on the training
// set.  Warm start: E_int,0 = rho c_v T exp(y_0), R_g,0 = E_g exp(y_g) - E_g
// - S_g.
//
// This header is included by rhd.cu after the single-grid machinery (pack,
// ensure_device, workspace, launch_mixed) it reuses.
#pragma once
#include "rhd_tc.cuh"

namespace rhd {
namespace mlp {

constexpr int kH = 128;       // hidden width
constexpr int kMaxGS = 64;    // largest N_g a surrogate supports
constexpr int kChunk = 1 << 20;  // cells per inference chunk
constexpr float kSigmaFloor = 1e-6f;

__host__ __device__ constexpr int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// ---- features / targets ----------------------------------------------------

__device__ __forceinline__ bool cell_T(const KParams &P, int64_t i, double &T) {
  const double rho = P.rho[i];
  const double m0 = P.mom[0][i], m1 = P.mom[1][i], m2 = P.mom[2][i];
  const double ke = 0.5 * (m0 * m0 + m1 * m1 + m2 * m2) / rho;
  T = (P.egas[i] - ke) / (rho * P.c_v);
  return rho > 0.0 && isfinite(T) && T > 0.0;
}

// Natural log of a positive normal double to FP32 accuracy without FP64
// instructions: ln(m 2^e) = e ln 2 + ln m, with m in [0.5, 1).
__device__ __forceinline__ float ln_f(double x) {
  int e;
  const float m = frexp_f(x, e);
  return (float)e * 0.69314718055994531f + __logf(m);
}

// The per-group features of a usable group energy e with flux (fx, fy, fz):
// ln(E_g / a_R T^4) held to [-700, 50] and |F_g| / (c E_g) held to 2, in FP32
// after the exact power-of-two scaling of E_g's exponent.
__device__ __forceinline__ void group_features(double e, double fx, double fy, double fz,
                                               float lnaT4, float c, float &fe, float &ff) {
  int ex;
  const float m = frexp_f(e, ex);
  const float ax = scaled_f(fx, ex), ay = scaled_f(fy, ex), az = scaled_f(fz, ex);
  fe = fminf(fmaxf((float)ex * 0.69314718055994531f + __logf(m) - lnaT4, -700.0f), 50.0f);
  ff = fminf(sqrtf(ax * ax + ay * ay + az * az) / (c * m), 2.0f);
}

// |v| / c and ln(c rho kappa0 dt) of a cell, in FP32 (rho v scaled by rho's exponent).
__device__ __forceinline__ void cell_scalar_features(const KParams &P, int64_t i, float &fv,
                                                     float &ft) {
  const double rho = P.rho[i];
  int er;
  const float mr = frexp_f(rho, er);
  const float a = scaled_f(P.mom[0][i], er), b = scaled_f(P.mom[1][i], er),
              c = scaled_f(P.mom[2][i], er);
  fv = sqrtf(a * a + b * b + c * c) / (mr * (float)P.c);
  const double k0 = P.kappa0 ? P.kappa0[i] : 1.0;
  const double tau = P.c * rho * k0 * P.dt;
  ft = usable_energy(tau) ? ln_f(tau) : -690.8f;  // ln 1e-300
}

// Raw features of one cell into f[0 .. 2G+4); false for an invalid cell.
// The per-group features are formed in FP32 after exact power-of-two
// scaling (the network consumes BF16; a guess needs no more).
__device__ __forceinline__ bool cell_features(const KParams &P, int64_t i, float *f) {
  const int G = P.G;
  double T;
  const bool ok = cell_T(P, i, T);
  if (!ok) {
    for (int k = 0; k < 2 * G + 4; ++k) f[k] = 0.0f;
    return false;
  }
  const double rho = P.rho[i];
  const float lnaT4 = ln_f(P.a_rad * T * T * T * T);
  f[0] = ln_f(rho);
  f[1] = ln_f(T);
  for (int g = 0; g < G; ++g) {
    const int64_t o = (int64_t)g * P.gs + i;
    const double e = P.erad[o];
    if (!usable_energy(e)) {  // empty (or denormal) group
      f[2 + g] = -700.0f;
      f[2 + G + g] = 0.0f;
      continue;
    }
    group_features(e, P.frad[0][o], P.frad[1][o], P.frad[2][o], lnaT4, (float)P.c, f[2 + g],
                   f[2 + G + g]);
  }
  cell_scalar_features(P, i, f[2 + 2 * G], f[3 + 2 * G]);
  return true;
}

__global__ void features_kernel(const __grid_constant__ KParams P, float *x, int64_t ldx) {
  float f[2 * kMaxGS + 4];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    cell_features(P, i, f);
    for (int k = 0; k < 2 * P.G + 4; ++k) x[i * ldx + k] = f[k];
  }
}

// Targets from the state before (A) and after (B) an update.
__global__ void targets_kernel(const __grid_constant__ KParams A, const __grid_constant__ KParams B,
                               float *y, int64_t ldy) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double Ta, Tb;
    const bool ok = cell_T(A, i, Ta) && cell_T(B, i, Tb);
    y[i * ldy] = ok ? (float)log(Tb / Ta) : 0.0f;
    for (int g = 0; g < A.G; ++g) {
      const int64_t o = (int64_t)g * A.gs + i;
      const double ea = A.erad[o], eb = B.erad[(int64_t)g * B.gs + i];
      y[i * ldy + 1 + g] = (ok && ea > 0.0 && eb > 0.0) ? (float)log(eb / ea) : 0.0f;
    }
  }
}

// Per-column mean and deviation of a row-major [n][cols] FP32 matrix (one
// block per column; FP64 sums).
__global__ void moments_kernel(const float *__restrict__ x, int64_t n, int cols, int64_t ld,
                               float *mean, float *sd) {
  const int col = blockIdx.x;
  double s = 0.0, s2 = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = x[r * ld + col];
    s += v;
    s2 += v * v;
  }
  __shared__ double a[256], b[256];
  a[threadIdx.x] = s;
  b[threadIdx.x] = s2;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h /= 2) {
    if ((int)threadIdx.x < h) {
      a[threadIdx.x] += a[threadIdx.x + h];
      b[threadIdx.x] += b[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = a[0] / (double)n;
    const double var = fmax(b[0] / (double)n - m * m, 0.0);
    mean[col] = (float)m;
    sd[col] = (float)fmax(sqrt(var), (double)kSigmaFloor);
  }
}

// ---- training ----------------------------------------------------------------

// Gather a batch: row j of the batch is sample (mult (first + j) + add) mod n.
// Writes the standardised inputs in BF16, row-major [B][ldxb] (columns past
// the feature count zero) and transposed [kin][B]; targets standardised FP32.
__global__ void batch_kernel(const float *__restrict__ x, const float *__restrict__ y, int64_t n,
                             int kin, int nout, int64_t first, int64_t mult, int64_t add,
                             int64_t B, const float *xm, const float *xs, const float *ym,
                             const float *ys, __nv_bfloat16 *xb, int64_t ldxb,
                             __nv_bfloat16 *xbt, float *yb) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < B;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = (int64_t)(((unsigned long long)mult * (unsigned long long)(first + j) +
                                 (unsigned long long)add) % (unsigned long long)n);
    for (int k = 0; k < ldxb; ++k) {
      const float v = k < kin ? (x[r * kin + k] - xm[k]) / xs[k] : 0.0f;
      const __nv_bfloat16 h = __float2bfloat16(v);
      xb[j * ldxb + k] = h;
      if (k < kin) xbt[(int64_t)k * B + j] = h;
    }
    for (int k = 0; k < nout; ++k) yb[j * nout + k] = (y[r * nout + k] - ym[k]) / ys[k];
  }
}

// dY = 2 (pred - y) / (B nout): FP32 (for the bias gradient), BF16 [B][ldd]
// and transposed BF16 [nout][B]; loss += mean squared error.
__global__ void loss_kernel(const float *__restrict__ pred, const float *__restrict__ yb, int64_t B,
                            int nout, float *dy, __nv_bfloat16 *dyb, int64_t lddy,
                            __nv_bfloat16 *dyt, float *loss) {
  const float scale = 2.0f / (float)(B * nout);
  float acc = 0.0f;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < B;
       j += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < lddy; ++k) {
      float d = 0.0f;
      if (k < nout) {
        const float e = pred[j * nout + k] - yb[j * nout + k];
        acc += e * e;
        d = scale * e;
        dy[j * nout + k] = d;
        dyt[(int64_t)k * B + j] = __float2bfloat16(d);
      }
      dyb[j * lddy + k] = __float2bfloat16(d);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc / (float)(B * nout));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * (z + k1 * z * z * z);
  const float t = tanhf(u);
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * k0 * (1.0f + 3.0f * k1 * z * z);
}

// dZ = dH * gelu'(Z), in place in dh (FP32), and as BF16 [B][kH].
__global__ void gelu_back_kernel(const float *__restrict__ z, float *dh, __nv_bfloat16 *dzb,
                                 int64_t count) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float d = dh[k] * gelu_grad(z[k]);
    dh[k] = d;
    dzb[k] = __float2bfloat16(d);
  }
}

// Column sums of a row-major [B][cols] FP32 matrix into out[cols] (one block per column).
__global__ void colsum_kernel(const float *__restrict__ a, int64_t B, int cols, float *out) {
  const int col = blockIdx.x;
  float s = 0.0f;
  for (int64_t r = threadIdx.x; r < B; r += blockDim.x) s += a[r * cols + col];
  __shared__ float t[256];
  t[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h /= 2) {
    if ((int)threadIdx.x < h) t[threadIdx.x] += t[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[col] = t[0];
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
}

// BF16 copies of W [rows][cols] (FP32): w [rows][ldw] and wt [cols][ldt]
// (zero-padded columns).
__global__ void publish_kernel(const float *__restrict__ W, int rows, int cols,
                               __nv_bfloat16 *w, int ldw, __nv_bfloat16 *wt, int ldt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < rows * ldw;
       k += gridDim.x * blockDim.x) {
    const int r = k / ldw, c = k % ldw;
    const float v = c < cols ? W[r * cols + c] : 0.0f;
    w[k] = __float2bfloat16(v);
    if (wt && c < cols) wt[(int64_t)c * ldt + r] = __float2bfloat16(v);
  }
  if (wt) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cols * ldt;
         k += gridDim.x * blockDim.x)
      if (k % ldt >= rows) wt[k] = __float2bfloat16(0.0f);
  }
}

// splitmix64-based uniform in [-1, 1) for the initial weights.
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t k) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (k + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0f - 1.0f;
}

__global__ void init_kernel(float *p, int64_t count, float scale, uint64_t seed, int64_t offset) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x)
    p[k] = scale * hash_uniform(seed, (uint64_t)(offset + k));
}

// ---- inference -----------------------------------------------------------------

// Standardised BF16 rows [m][ldx] from raw FP32 features x [m][kin].
__global__ void standardize_kernel(const float *__restrict__ x, int64_t m, int kin,
                                   const float *xm, const float *xs, __nv_bfloat16 *xb,
                                   int64_t ldx) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < ldx; ++k)
      xb[j * ldx + k] = __float2bfloat16(k < kin ? (x[j * kin + k] - xm[k]) / xs[k] : 0.0f);
}

// y = y * sd + mean, per column, in place ([m][nout]).
__global__ void destandardize_kernel(float *y, int64_t m, int nout, const float *ym,
                                     const float *ys) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m * nout;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(k % nout);
    y[k] = y[k] * ys[c] + ym[c];
  }
}

}  // namespace mlp
}  // namespace rhd

#include "rhd_mlp_fused.cuh"

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct rhd_surrogate {
  int device = -1;
  int G = 0, kin = 0, kpad = 0, nout = 0, npad = 0;
  int64_t nparam = 0;
  int64_t off_w[4] = {0, 0, 0, 0}, off_b[4] = {0, 0, 0, 0};
  int in[4] = {0, 0, 0, 0}, out[4] = {0, 0, 0, 0};
  float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
  int64_t step = 0;
  __nv_bfloat16 *w[4] = {nullptr, nullptr, nullptr, nullptr};
  __nv_bfloat16 *wt[4] = {nullptr, nullptr, nullptr, nullptr};
  float *norm = nullptr;  // x_mean [kin], x_sd [kin], y_mean [nout], y_sd [nout]
  unsigned *err = nullptr;
  int wait_test = 0;  // rhd_surrogate_test_wait_timeout
  // training buffers (capacity cap_b rows)
  int64_t cap_b = 0;
  void *tbuf = nullptr;
  // inference buffers (capacity kChunk rows)
  void *ibuf = nullptr;
};

namespace rhd {
namespace {

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

float *xm(rhd_surrogate *s) { return s->norm; }
float *xsd(rhd_surrogate *s) { return s->norm + s->kin; }
float *ym(rhd_surrogate *s) { return s->norm + 2 * s->kin; }
float *ysd(rhd_surrogate *s) { return s->norm + 2 * s->kin + s->nout; }

int blocks_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

int publish(rhd_surrogate *s, cudaStream_t st) {
  for (int l = 0; l < 4; ++l) {
    const int ldw = (int)mlp::round8(s->in[l]);
    const int ldt = (int)mlp::round8(s->out[l]);
    mlp::publish_kernel<<<blocks_for((int64_t)s->out[l] * ldw, 256), 256, 0, st>>>(
        s->params + s->off_w[l], s->out[l], s->in[l], s->w[l], ldw, l > 0 ? s->wt[l] : nullptr,
        ldt);
  }
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

// Training views into tbuf for a batch of B rows.
struct TrainBufs {
  __nv_bfloat16 *xb, *xbt, *h[3], *ht, *dyb, *dyt, *dzb, *dzt;
  float *yb, *z[3], *pred, *dy, *dh;
};

int64_t train_bytes(const rhd_surrogate *s, int64_t B) {
  const int64_t b16 = 2, b32 = 4, H = mlp::kH;
  return align256(B * s->kpad * b16) + align256((int64_t)s->kpad * B * b16) +
         3 * align256(B * H * b16) + align256(H * B * b16) + align256(B * s->npad * b16) +
         align256((int64_t)s->npad * B * b16) + align256(B * H * b16) + align256(H * B * b16) +
         align256(B * s->nout * b32) + 3 * align256(B * H * b32) + align256(B * s->nout * b32) +
         align256(B * s->nout * b32) + align256(B * H * b32);
}

TrainBufs train_views(rhd_surrogate *s, int64_t B) {
  char *p = (char *)s->tbuf;
  const int64_t H = mlp::kH;
  auto take = [&](int64_t bytes) {
    char *q = p;
    p += align256(bytes);
    return q;
  };
  TrainBufs t;
  t.xb = (__nv_bfloat16 *)take(B * s->kpad * 2);
  t.xbt = (__nv_bfloat16 *)take((int64_t)s->kpad * B * 2);
  for (int l = 0; l < 3; ++l) t.h[l] = (__nv_bfloat16 *)take(B * H * 2);
  t.ht = (__nv_bfloat16 *)take(H * B * 2);
  t.dyb = (__nv_bfloat16 *)take(B * s->npad * 2);
  t.dyt = (__nv_bfloat16 *)take((int64_t)s->npad * B * 2);
  t.dzb = (__nv_bfloat16 *)take(B * H * 2);
  t.dzt = (__nv_bfloat16 *)take(H * B * 2);
  t.yb = (float *)take(B * s->nout * 4);
  for (int l = 0; l < 3; ++l) t.z[l] = (float *)take(B * H * 4);
  t.pred = (float *)take(B * s->nout * 4);
  t.dy = (float *)take(B * s->nout * 4);
  t.dh = (float *)take(B * H * 4);
  return t;
}

int ensure_train(rhd_surrogate *s, int64_t B) {
  if (B <= s->cap_b) return RHD_OK;
  if (s->tbuf) cudaFree(s->tbuf);
  s->tbuf = nullptr;
  s->cap_b = 0;
  if (cudaMalloc(&s->tbuf, (size_t)train_bytes(s, B)) != cudaSuccess) return RHD_ENOMEM;
  s->cap_b = B;
  return RHD_OK;
}

tc::GemmArgs gemm_args(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *Bm, int64_t ldb,
                       int64_t M, int64_t N, int64_t K, float *D, int64_t ldd, int epi,
                       const float *bias, __nv_bfloat16 *H, int64_t ldh, const rhd_surrogate *s) {
  tc::GemmArgs g{};
  g.A = A;
  g.lda = lda;
  g.B = Bm;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.D = D;
  g.ldd = ldd;
  g.epi = epi;
  g.bias = bias;
  g.H = H;
  g.ldh = ldh;
  g.err = s->err;
  g.wait_test = s->wait_test;
  return g;
}

// Forward + backward of one batch already in t (xb, xbt, yb); gradients into
// s->grads, loss (if non-null) accumulated.
int forward_backward(rhd_surrogate *s, const TrainBufs &t, int64_t B, float *loss,
                     cudaStream_t st) {
  const int64_t H = mlp::kH;
  cudaError_t e = cudaSuccess;
  auto run = [&](const tc::GemmArgs &g) {
    if (e == cudaSuccess) e = tc::gemm(g, st);
  };
  // forward
  run(gemm_args(t.xb, s->kpad, s->w[0], s->kpad, B, H, s->kin, t.z[0], H, tc::kEpiBiasGelu,
                s->params + s->off_b[0], t.h[0], H, s));
  for (int l = 1; l < 3; ++l)
    run(gemm_args(t.h[l - 1], H, s->w[l], H, B, H, H, t.z[l], H, tc::kEpiBiasGelu,
                  s->params + s->off_b[l], t.h[l], H, s));
  run(gemm_args(t.h[2], H, s->w[3], H, B, s->nout, H, t.pred, s->nout, tc::kEpiBias,
                s->params + s->off_b[3], nullptr, 0, s));
  if (e != cudaSuccess) return RHD_ECUDA;
  mlp::loss_kernel<<<blocks_for(B, 256), 256, 0, st>>>(t.pred, t.yb, B, s->nout, t.dy, t.dyb,
                                                       s->npad, t.dyt, loss);
  mlp::colsum_kernel<<<s->nout, 256, 0, st>>>(t.dy, B, s->nout, s->grads + s->off_b[3]);
  // layer 4: dW4 = dY^T H3, dH3 = dY W4
  e = tc::transpose(t.h[2], B, H, H, t.ht, B, st);
  run(gemm_args(t.dyt, B, t.ht, B, s->nout, H, B, s->grads + s->off_w[3], H, tc::kEpiStore,
                nullptr, nullptr, 0, s));
  run(gemm_args(t.dyb, s->npad, s->wt[3], s->npad, B, H, s->nout, t.dh, H, tc::kEpiStore,
                nullptr, nullptr, 0, s));
  for (int l = 2; l >= 0; --l) {
    if (e != cudaSuccess) return RHD_ECUDA;
    mlp::gelu_back_kernel<<<blocks_for(B * H, 256), 256, 0, st>>>(t.z[l], t.dh, t.dzb, B * H);
    mlp::colsum_kernel<<<(unsigned)H, 256, 0, st>>>(t.dh, B, (int)H, s->grads + s->off_b[l]);
    if (e == cudaSuccess) e = tc::transpose(t.dzb, B, H, H, t.dzt, B, st);
    if (l > 0) {
      // dW_l = dZ^T H_{l-1}; dH_{l-1} = dZ W_l
      if (e == cudaSuccess) e = tc::transpose(t.h[l - 1], B, H, H, t.ht, B, st);
      run(gemm_args(t.dzt, B, t.ht, B, H, H, B, s->grads + s->off_w[l], H, tc::kEpiStore,
                    nullptr, nullptr, 0, s));
      run(gemm_args(t.dzb, H, s->wt[l], H, B, H, H, t.dh, H, tc::kEpiStore, nullptr, nullptr, 0,
                    s));
    } else {
      // dW_1 = dZ^T X
      run(gemm_args(t.dzt, B, t.xbt, B, H, s->kin, B, s->grads + s->off_w[0], s->kin,
                    tc::kEpiStore, nullptr, nullptr, 0, s));
    }
  }
  return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? RHD_OK : RHD_ECUDA;
}

int load_batch(rhd_surrogate *s, const TrainBufs &t, const float *x, const float *y, int64_t n,
               int64_t first, int64_t B, int64_t mult, int64_t add, cudaStream_t st) {
  mlp::batch_kernel<<<blocks_for(B, 128), 128, 0, st>>>(x, y, n, s->kin, s->nout, first, mult,
                                                        add, B, xm(s), xsd(s), ym(s), ysd(s),
                                                        t.xb, s->kpad, t.xbt, t.yb);
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

// Inference buffers: features [kChunk][kpad], two hidden [kChunk][kH], output [kChunk][nout].
int ensure_infer(rhd_surrogate *s) {
  if (s->ibuf) return RHD_OK;
  const int64_t C = mlp::kChunk;
  const size_t bytes = (size_t)(align256(C * s->kpad * 2) + 2 * align256(C * mlp::kH * 2) +
                                align256(C * s->nout * 4));
  if (cudaMalloc(&s->ibuf, bytes) != cudaSuccess) return RHD_ENOMEM;
  return RHD_OK;
}

struct InferBufs {
  __nv_bfloat16 *xb, *h0, *h1;
  float *y;
};

InferBufs infer_views(rhd_surrogate *s) {
  const int64_t C = mlp::kChunk, H = mlp::kH;
  char *p = (char *)s->ibuf;
  InferBufs b;
  b.xb = (__nv_bfloat16 *)p;
  p += align256(C * s->kpad * 2);
  b.h0 = (__nv_bfloat16 *)p;
  p += align256(C * H * 2);
  b.h1 = (__nv_bfloat16 *)p;
  p += align256(C * H * 2);
  b.y = (float *)p;
  return b;
}

// The network on the m (<= kChunk) standardised rows in b.xb: standardised
// outputs into y [m][nout].
int infer_rows(rhd_surrogate *s, const InferBufs &b, int64_t m, float *y, cudaStream_t st) {
  const int64_t H = mlp::kH;
  cudaError_t e = tc::gemm(gemm_args(b.xb, s->kpad, s->w[0], s->kpad, m, H, s->kin, nullptr, H,
                                     tc::kEpiBiasGelu, s->params + s->off_b[0], b.h0, H, s),
                           st);
  if (e == cudaSuccess)
    e = tc::gemm(gemm_args(b.h0, H, s->w[1], H, m, H, H, nullptr, H, tc::kEpiBiasGelu,
                           s->params + s->off_b[1], b.h1, H, s),
                 st);
  if (e == cudaSuccess)
    e = tc::gemm(gemm_args(b.h1, H, s->w[2], H, m, H, H, nullptr, H, tc::kEpiBiasGelu,
                           s->params + s->off_b[2], b.h0, H, s),
                 st);
  if (e == cudaSuccess)
    e = tc::gemm(gemm_args(b.h0, H, s->w[3], H, m, s->nout, H, y, s->nout, tc::kEpiBias,
                           s->params + s->off_b[3], nullptr, 0, s),
                 st);
  return e == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

// The fused inference (rhd_mlp_fused.cuh) over all cells of kp into W.
int launch_fused(rhd_surrogate *s, const KParams &kp, const WarmOut &W, bool full, int sms,
                 cudaStream_t st) {
  mlp::FusedNet N;
  for (int l = 0; l < 4; ++l) {
    N.w[l] = s->w[l];
    N.b[l] = s->params + s->off_b[l];
  }
  N.xm = xm(s);
  N.xs = xsd(s);
  N.ym = ym(s);
  N.ys = ysd(s);
  N.kin = s->kin;
  N.nout = s->nout;
  N.k1 = mlp::round16(s->kin);
  N.n4 = mlp::round16(s->nout);
  N.full = full ? 1 : 0;
  N.err = s->err;
  const size_t smem = mlp::fused_bytes(N.k1, N.n4);
  if (allow_smem<mlp::infer_fused_kernel>(smem) != cudaSuccess) return RHD_ECUDA;
  const int64_t tiles = (kp.n + tc::kTileM - 1) / tc::kTileM;
  const int64_t pairs = (tiles + mlp::kFusedGroups - 1) / mlp::kFusedGroups;
  const int blocks = (int)(pairs < sms ? pairs : sms);
  if (blocks > 0)
    timed_launch(RHD_KERNEL_INFERENCE, st, [&] {
      mlp::infer_fused_kernel<<<blocks, 128 * mlp::kFusedGroups, smem, st>>>(kp, N, W);
    });
  if (kp.count) t_infer_cells += (unsigned long long)kp.n;
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

// Parameters of the network for n_groups groups: (2 N_g + 4) -> H -> H -> H
// -> N_g + 1, weights and biases.
int64_t param_count(int n_groups) {
  const int64_t H = mlp::kH, kin = 2 * (int64_t)n_groups + 4, nout = (int64_t)n_groups + 1;
  return kin * H + H + 2 * (H * H + H) + H * nout + nout;
}

int check_surrogate(const rhd_surrogate *s) {
  if (!s) return RHD_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RHD_ECUDA;
  return dev == s->device ? RHD_OK : RHD_EINVAL;
}

}  // namespace
}  // namespace rhd

extern "C" int rhd_surrogate_create(int32_t n_groups, uint64_t seed, rhd_surrogate_t **out) {
  if (!out || n_groups < 1 || n_groups > rhd::mlp::kMaxGS) return n_groups > rhd::mlp::kMaxGS ? RHD_ESIZE : RHD_EINVAL;
  int sms = 0;
  int rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  rhd_surrogate *s = new (std::nothrow) rhd_surrogate();
  if (!s) return RHD_ENOMEM;
  cudaGetDevice(&s->device);
  const int H = rhd::mlp::kH;
  s->G = n_groups;
  s->kin = 2 * n_groups + 4;
  s->kpad = (int)rhd::mlp::round8(s->kin);
  s->nout = n_groups + 1;
  s->npad = (int)rhd::mlp::round8(s->nout);
  const int ins[4] = {s->kin, H, H, H}, outs[4] = {H, H, H, s->nout};
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    s->in[l] = ins[l];
    s->out[l] = outs[l];
    s->off_w[l] = off;
    off += (int64_t)ins[l] * outs[l];
    s->off_b[l] = off;
    off += outs[l];
  }
  s->nparam = off;
  bool ok = cudaMalloc(&s->params, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&s->grads, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&s->am, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&s->av, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&s->norm, sizeof(float) * 2 * (s->kin + s->nout)) == cudaSuccess &&
            cudaMalloc(&s->err, sizeof(unsigned)) == cudaSuccess;
  for (int l = 0; l < 4 && ok; ++l) {
    ok = cudaMalloc(&s->w[l], 2 * (size_t)outs[l] * rhd::mlp::round8(ins[l])) == cudaSuccess &&
         cudaMalloc(&s->wt[l], 2 * (size_t)ins[l] * rhd::mlp::round8(outs[l])) == cudaSuccess;
  }
  if (!ok) {
    rhd_surrogate_destroy(s);
    return RHD_ENOMEM;
  }
  // He-style uniform initial weights (last layer scaled down), zero biases,
  // identity standardisation, zero Adam moments
  cudaMemset(s->params, 0, sizeof(float) * off);
  cudaMemset(s->am, 0, sizeof(float) * off);
  cudaMemset(s->av, 0, sizeof(float) * off);
  cudaMemset(s->err, 0, sizeof(unsigned));
  for (int l = 0; l < 4; ++l) {
    const float scale = sqrtf(6.0f / (float)ins[l]) * (l == 3 ? 0.1f : 1.0f);
    const int64_t cnt = (int64_t)ins[l] * outs[l];
    rhd::mlp::init_kernel<<<rhd::blocks_for(cnt, 256), 256>>>(s->params + s->off_w[l], cnt, scale,
                                                              seed, s->off_w[l]);
  }
  {
    float *h = new (std::nothrow) float[2 * (s->kin + s->nout)];
    if (!h) {
      rhd_surrogate_destroy(s);
      return RHD_ENOMEM;
    }
    for (int k = 0; k < s->kin; ++k) {
      h[k] = 0.0f;
      h[s->kin + k] = 1.0f;
    }
    for (int k = 0; k < s->nout; ++k) {
      h[2 * s->kin + k] = 0.0f;
      h[2 * s->kin + s->nout + k] = 1.0f;
    }
    cudaMemcpy(s->norm, h, sizeof(float) * 2 * (s->kin + s->nout), cudaMemcpyHostToDevice);
    delete[] h;
  }
  rc = rhd::publish(s, 0);
  if (rc == RHD_OK && cudaDeviceSynchronize() != cudaSuccess) rc = RHD_ECUDA;
  if (rc != RHD_OK) {
    rhd_surrogate_destroy(s);
    return rc;
  }
  *out = s;
  return RHD_OK;
}

extern "C" int rhd_surrogate_destroy(rhd_surrogate_t *s) {
  if (!s) return RHD_EINVAL;
  cudaDeviceSynchronize();
  cudaFree(s->params);
  cudaFree(s->grads);
  cudaFree(s->am);
  cudaFree(s->av);
  cudaFree(s->norm);
  cudaFree(s->err);
  for (int l = 0; l < 4; ++l) {
    cudaFree(s->w[l]);
    cudaFree(s->wt[l]);
  }
  cudaFree(s->tbuf);
  cudaFree(s->ibuf);
  delete s;
  return RHD_OK;
}

extern "C" int rhd_surrogate_dims(const rhd_surrogate_t *s, int32_t *n_features,
                                  int32_t *n_outputs, int64_t *n_params) {
  if (!s || !n_features || !n_outputs || !n_params) return RHD_EINVAL;
  *n_features = s->kin;
  *n_outputs = s->nout;
  *n_params = s->nparam;
  return RHD_OK;
}

extern "C" int rhd_surrogate_features(const rhd_surrogate_t *s, const rhd_state_t *state,
                                      const rhd_groups_t *groups,
                                      const rhd_opacity_law_t *opacity_law, double dt,
                                      int64_t n_cells, float *x, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  static thread_local rhd::KParams kp;
  rc = rhd::pack(state, groups, opacity_law, dt, n_cells, &kp);
  if (rc != RHD_OK) return rc;
  if (groups->n_groups != s->G) return RHD_EINVAL;
  if (n_cells == 0) return RHD_OK;
  if (!x) return RHD_EINVAL;
  rhd::mlp::features_kernel<<<rhd::blocks_for(n_cells, 128), 128, 0, (cudaStream_t)stream>>>(
      kp, x, s->kin);
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

extern "C" int rhd_surrogate_targets(const rhd_surrogate_t *s, const rhd_state_t *before,
                                     const rhd_state_t *after, const rhd_groups_t *groups,
                                     const rhd_opacity_law_t *opacity_law, double dt,
                                     int64_t n_cells, float *y, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  static thread_local rhd::KParams ka, kb;
  rc = rhd::pack(before, groups, opacity_law, dt, n_cells, &ka);
  if (rc == RHD_OK) rc = rhd::pack(after, groups, opacity_law, dt, n_cells, &kb);
  if (rc != RHD_OK) return rc;
  if (groups->n_groups != s->G) return RHD_EINVAL;
  if (n_cells == 0) return RHD_OK;
  if (!y) return RHD_EINVAL;
  rhd::mlp::targets_kernel<<<rhd::blocks_for(n_cells, 128), 128, 0, (cudaStream_t)stream>>>(
      ka, kb, y, s->nout);
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

extern "C" int rhd_surrogate_fit_normalization(rhd_surrogate_t *s, const float *x, const float *y,
                                               int64_t n, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  if (!x || !y || n < 2) return RHD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rhd::mlp::moments_kernel<<<s->kin, 256, 0, st>>>(x, n, s->kin, s->kin, rhd::xm(s), rhd::xsd(s));
  rhd::mlp::moments_kernel<<<s->nout, 256, 0, st>>>(y, n, s->nout, s->nout, rhd::ym(s),
                                                    rhd::ysd(s));
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

extern "C" int rhd_surrogate_params(rhd_surrogate_t *s, float *params, float *normalization,
                                    int32_t set, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t pb = sizeof(float) * s->nparam, nb = sizeof(float) * 2 * (s->kin + s->nout);
  if (set) {
    if (params && cudaMemcpyAsync(s->params, params, pb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return RHD_ECUDA;
    if (normalization &&
        cudaMemcpyAsync(s->norm, normalization, nb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return RHD_ECUDA;
    if (params) {
      cudaMemsetAsync(s->am, 0, pb, st);
      cudaMemsetAsync(s->av, 0, pb, st);
      s->step = 0;
      return rhd::publish(s, st);
    }
    return RHD_OK;
  }
  if (params && cudaMemcpyAsync(params, s->params, pb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return RHD_ECUDA;
  if (normalization &&
      cudaMemcpyAsync(normalization, s->norm, nb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return RHD_ECUDA;
  return RHD_OK;
}

extern "C" int rhd_surrogate_loss_grad(rhd_surrogate_t *s, const float *x, const float *y,
                                       int64_t n, float *loss, float *grad, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  if (!x || !y || n < 1 || n % 8) return RHD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rc = rhd::ensure_train(s, n);
  if (rc != RHD_OK) return rc;
  const rhd::TrainBufs t = rhd::train_views(s, n);
  rc = rhd::load_batch(s, t, x, y, n, 0, n, 1, 0, st);
  if (rc == RHD_OK && loss) rc = cudaMemsetAsync(loss, 0, sizeof(float), st) == cudaSuccess ? RHD_OK : RHD_ECUDA;
  if (rc == RHD_OK) rc = rhd::forward_backward(s, t, n, loss, st);
  if (rc == RHD_OK && grad &&
      cudaMemcpyAsync(grad, s->grads, sizeof(float) * s->nparam, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    rc = RHD_ECUDA;
  return rc;
}

extern "C" int rhd_surrogate_train_step(rhd_surrogate_t *s, const float *x, const float *y,
                                        int64_t n_rows, int64_t first, int64_t batch,
                                        int64_t perm_mult, int64_t perm_add, float lr,
                                        float *loss, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  if (!x || !y || n_rows < 1 || batch < 8 || batch % 8 || perm_mult < 1 || perm_add < 0 ||
      !(lr > 0.0f))
    return RHD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rc = rhd::ensure_train(s, batch);
  if (rc != RHD_OK) return rc;
  const rhd::TrainBufs t = rhd::train_views(s, batch);
  rc = rhd::load_batch(s, t, x, y, n_rows, first, batch, perm_mult, perm_add, st);
  if (rc == RHD_OK) rc = rhd::forward_backward(s, t, batch, loss, st);
  if (rc != RHD_OK) return rc;
  ++s->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)s->step), c2 = 1.0f - powf(b2, (float)s->step);
  rhd::mlp::adam_kernel<<<rhd::blocks_for(s->nparam, 256), 256, 0, st>>>(
      s->params, s->grads, s->am, s->av, s->nparam, lr, b1, b2, 1e-8f, c1, c2);
  return rhd::publish(s, st);
}

extern "C" int rhd_surrogate_predict(rhd_surrogate_t *s, const float *x, int64_t n, float *y,
                                     void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  if (n == 0) return RHD_OK;
  if (!x || !y || n < 0) return RHD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rc = rhd::ensure_infer(s);
  if (rc != RHD_OK) return rc;
  const rhd::InferBufs b = rhd::infer_views(s);
  for (int64_t c0 = 0; c0 < n && rc == RHD_OK; c0 += rhd::mlp::kChunk) {
    const int64_t m = n - c0 < rhd::mlp::kChunk ? n - c0 : rhd::mlp::kChunk;
    rhd::mlp::standardize_kernel<<<rhd::blocks_for(m, 128), 128, 0, st>>>(
        x + c0 * s->kin, m, s->kin, rhd::xm(s), rhd::xsd(s), b.xb, s->kpad);
    rc = rhd::infer_rows(s, b, m, y + c0 * s->nout, st);
    if (rc == RHD_OK)
      rhd::mlp::destandardize_kernel<<<rhd::blocks_for(m * s->nout, 256), 256, 0, st>>>(
          y + c0 * s->nout, m, s->nout, rhd::ym(s), rhd::ysd(s));
  }
  if (rc == RHD_OK && cudaGetLastError() != cudaSuccess) rc = RHD_ECUDA;
  return rc;
}

extern "C" int rhd_surrogate_test_wait_timeout(rhd_surrogate_t *s, int32_t on) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  s->wait_test = on ? 1 : 0;
  return RHD_OK;
}

extern "C" int rhd_surrogate_error(rhd_surrogate_t *s, int32_t *flag) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  if (!flag) return RHD_EINVAL;
  unsigned h = 0;
  if (cudaMemcpy(&h, s->err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return RHD_ECUDA;
  *flag = (int32_t)h;
  return RHD_OK;
}

extern "C" int rhd_source_update_warm(rhd_surrogate_t *s, rhd_state_t *state,
                                      const rhd_groups_t *groups,
                                      const rhd_opacity_law_t *opacity_law, double dt,
                                      int64_t n_cells, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  static thread_local rhd::KParams kp;
  rc = rhd::pack(state, groups, opacity_law, dt, n_cells, &kp);
  if (rc != RHD_OK) return rc;
  if (groups->n_groups != s->G) return RHD_EINVAL;
  if (n_cells == 0) return RHD_OK;
  int sms = 0;
  rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  rhd::WarmOut wo;
  rhd::WarmStart wi;
  rc = rhd::workspace(kp.n, kp.G, &wo, &wi);
  if (rc != RHD_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // the FP32 passes read only E_int,0 and R_g,0; the FP64 passes started
  // directly (FP64 form, free slopes) also take rho v, F_g and the iterations
  const bool full = state->precision == RHD_FP64 || kp.mode == RHD_PPL_FREE;
  rc = rhd::launch_fused(s, kp, wo, full, sms, st);
  if (rc != RHD_OK) return rc;
  return rhd::launch_warm(kp, state->precision, wo, wi, sms, st);
}

extern "C" int rhd_surrogate_warm_start(rhd_surrogate_t *s, const rhd_state_t *state,
                                        const rhd_groups_t *groups,
                                        const rhd_opacity_law_t *opacity_law, double dt,
                                        int64_t n_cells, double *eint, float *r, void *stream) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  static thread_local rhd::KParams kp;
  rc = rhd::pack(state, groups, opacity_law, dt, n_cells, &kp);
  if (rc != RHD_OK) return rc;
  if (groups->n_groups != s->G) return RHD_EINVAL;
  if (n_cells == 0) return RHD_OK;
  if (!eint || !r) return RHD_EINVAL;
  int sms = 0;
  rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  rhd::WarmOut wo{eint, nullptr, r, nullptr, nullptr};
  return rhd::launch_fused(s, kp, wo, false, sms, (cudaStream_t)stream);
}

// ---- saving and loading a network ------------------------------------------
namespace rhd {
namespace {
constexpr char kMlpMagic[8] = {'R', 'H', 'D', 'M', 'L', 'P', '1', '\0'};
// the same, followed by the Adam moments and step count (rhd_surrogate_checkpoint)
constexpr char kMlpMagicTrain[8] = {'R', 'H', 'D', 'M', 'L', 'P', '2', '\0'};

struct MlpHeader {
  char magic[8];
  int32_t n_groups, n_features, n_outputs;
  int32_t pad;
  int64_t n_params;
};
static_assert(sizeof(MlpHeader) == 32, "file header");
}  // namespace
}  // namespace rhd

extern "C" int rhd_surrogate_save(rhd_surrogate_t *s, const char *path) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  if (!path) return RHD_EINVAL;
  const size_t np = (size_t)s->nparam, nn = 2 * (size_t)(s->kin + s->nout);
  std::vector<float> buf(np + nn);
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(buf.data(), s->params, sizeof(float) * np, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + np, s->norm, sizeof(float) * nn, cudaMemcpyDeviceToHost) != cudaSuccess)
    return RHD_ECUDA;
  rhd::MlpHeader h{};
  std::memcpy(h.magic, rhd::kMlpMagic, 8);
  h.n_groups = s->G;
  h.n_features = s->kin;
  h.n_outputs = s->nout;
  h.n_params = s->nparam;
  FILE *f = std::fopen(path, "wb");
  if (!f) return RHD_EIO;
  const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                  std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  return (std::fclose(f) == 0 && ok) ? RHD_OK : RHD_EIO;
}

extern "C" int rhd_surrogate_checkpoint(rhd_surrogate_t *s, const char *path) {
  int rc = rhd::check_surrogate(s);
  if (rc != RHD_OK) return rc;
  if (!path) return RHD_EINVAL;
  const size_t np = (size_t)s->nparam, nn = 2 * (size_t)(s->kin + s->nout);
  std::vector<float> buf(3 * np + nn);
  const cudaMemcpyKind D2H = cudaMemcpyDeviceToHost;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(buf.data(), s->params, sizeof(float) * np, D2H) != cudaSuccess ||
      cudaMemcpy(buf.data() + np, s->norm, sizeof(float) * nn, D2H) != cudaSuccess ||
      cudaMemcpy(buf.data() + np + nn, s->am, sizeof(float) * np, D2H) != cudaSuccess ||
      cudaMemcpy(buf.data() + 2 * np + nn, s->av, sizeof(float) * np, D2H) != cudaSuccess)
    return RHD_ECUDA;
  rhd::MlpHeader h{};
  std::memcpy(h.magic, rhd::kMlpMagicTrain, 8);
  h.n_groups = s->G;
  h.n_features = s->kin;
  h.n_outputs = s->nout;
  h.n_params = s->nparam;
  const int64_t step = s->step;
  FILE *f = std::fopen(path, "wb");
  if (!f) return RHD_EIO;
  const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                  std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size() &&
                  std::fwrite(&step, sizeof(step), 1, f) == 1;
  return (std::fclose(f) == 0 && ok) ? RHD_OK : RHD_EIO;
}

extern "C" int rhd_surrogate_load(const char *path, rhd_surrogate_t **out) {
  if (!path || !out) return RHD_EINVAL;
  *out = nullptr;
  FILE *f = std::fopen(path, "rb");
  if (!f) return RHD_EIO;
  rhd::MlpHeader h{};
  const bool head_ok = std::fread(&h, sizeof(h), 1, f) == 1 &&
                       (std::memcmp(h.magic, rhd::kMlpMagic, 8) == 0 ||
                        std::memcmp(h.magic, rhd::kMlpMagicTrain, 8) == 0) &&
                       h.n_groups >= 1 &&
                       h.n_groups <= rhd::mlp::kMaxGS && h.n_params > 0 &&
                       h.n_features == 2 * h.n_groups + 4 && h.n_outputs == h.n_groups + 1;
  if (!head_ok) {
    std::fclose(f);
    return RHD_EIO;
  }
  const bool train = std::memcmp(h.magic, rhd::kMlpMagicTrain, 8) == 0;
  // the parameter count is fixed by the group count: a header that says
  // otherwise is corrupt (and must not size the buffer below)
  if ((int64_t)h.n_params != rhd::param_count(h.n_groups)) {
    std::fclose(f);
    return RHD_EIO;
  }
  const size_t np = (size_t)h.n_params, nn = 2 * (size_t)(h.n_features + h.n_outputs);
  std::vector<float> buf(np + nn + (train ? 2 * np : 0));
  int64_t step = 0;
  const bool body_ok = std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size() &&
                       (!train || (std::fread(&step, sizeof(step), 1, f) == 1 && step >= 0)) &&
                       std::fgetc(f) == EOF;
  std::fclose(f);
  if (!body_ok) return RHD_EIO;
  rhd_surrogate_t *s = nullptr;
  int rc = rhd_surrogate_create(h.n_groups, 0, &s);
  if (rc != RHD_OK) return rc;
  if (s->nparam != h.n_params || s->kin != h.n_features || s->nout != h.n_outputs) {
    rhd_surrogate_destroy(s);
    return RHD_EIO;
  }
  const cudaMemcpyKind H2D = cudaMemcpyHostToDevice;
  const bool moments_ok =
      train ? (cudaMemcpy(s->am, buf.data() + np + nn, sizeof(float) * np, H2D) == cudaSuccess &&
               cudaMemcpy(s->av, buf.data() + 2 * np + nn, sizeof(float) * np, H2D) == cudaSuccess)
            : (cudaMemset(s->am, 0, sizeof(float) * np) == cudaSuccess &&
               cudaMemset(s->av, 0, sizeof(float) * np) == cudaSuccess);
  if (cudaMemcpy(s->params, buf.data(), sizeof(float) * np, H2D) != cudaSuccess ||
      cudaMemcpy(s->norm, buf.data() + np, sizeof(float) * nn, H2D) != cudaSuccess || !moments_ok) {
    rhd_surrogate_destroy(s);
    return RHD_ECUDA;
  }
  s->step = train ? step : 0;
  rc = rhd::publish(s, nullptr);
  if (rc == RHD_OK && cudaDeviceSynchronize() != cudaSuccess) rc = RHD_ECUDA;
  if (rc != RHD_OK) {
    rhd_surrogate_destroy(s);
    return rc;
  }
  *out = s;
  return RHD_OK;
}
