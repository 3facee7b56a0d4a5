// mlp.cu -- learned warm start of the Z0 solve (not part of the paper, whose
// solve starts GMRES from the previous data, section 2.6).
//
// For every RWG edge (and right-hand side) a small odd perceptron predicts
// the correction of the cubic time extrapolation of the edge's current from
// local data: the past four currents of the edge and of its four RWG
// neighbours (orientation-signed) and the Jacobi-scaled right-hand sides
// b_j / Z0_jj of the same five edges, all divided by their RMS.  Division by
// the RMS and the oddness of the network (tanh, no biases) keep the
// prediction linear in the overall scale and sign of the data, as the march
// itself is.  The Z0 solve still runs to its tolerance from whichever of the
// prediction and the plain extrapolation has the smaller FP64 residual, so
// the network changes the work, never the result.
//
// Kernels (all FP32 arithmetic on FP32 parameters, features formed in FP64):
//   k_mlp_infer   features + forward pass for every (edge, RHS), writes x0;
//   k_mlp_record  features + target of the step just solved, appended to the
//                 training set;
//   k_mlp_train   forward and backward pass of one minibatch, 128 samples per
//                 block: activations and their gradients in shared memory,
//                 weight gradients as block-level sums over the samples,
//                 one atomic add per parameter per block;
//   k_mlp_adam    Adam update, then the gradient is cleared.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "internal.h"

namespace tdbem {

constexpr int kF = TDBEM_MLP_FEATURES, kH = TDBEM_MLP_WIDTH, kNP = TDBEM_MLP_NPARAM;
constexpr int kTB = 128;      // samples per training block
constexpr int kHS = kH + 1;   // padded row stride of per-sample activations in shared memory

struct FeatArgs {
  const double* ring;      // [ne][L][R]
  const double* b;         // [ne][R] right-hand side of this step
  const double* inv_diag;  // [ne] 1 / Z0_ii
  const int32_t* nb;       // [ne][4] neighbour edges
  const int8_t* nbs;       // [ne][4] orientation signs
  int64_t ne;
  int32_t L, R, alpha;
};

// J_j^{beta} of right-hand side r from the ring (zero before step 0)
__device__ __forceinline__ double hist(const FeatArgs& a, int64_t j, int r, int beta) {
  return beta >= 0 ? a.ring[(j * a.L + (beta & (a.L - 1))) * a.R + r] : 0.0;
}

// Features of (edge i, RHS r) for the solve of J^{alpha-1}: x = f / s (float),
// the scale s and the cubic extrapolation xc.
__device__ __forceinline__ void features(const FeatArgs& a, int64_t i, int r, float* x, double& s, double& xc) {
  double f[kF];
  const int b1 = a.alpha - 2;  // J^{alpha-2}, the newest known current
  for (int k = 0; k < 4; ++k) f[k] = hist(a, i, r, b1 - k);
  for (int n = 0; n < 4; ++n) {
    const int64_t j = a.nb[4 * i + n];
    const double sg = (double)a.nbs[4 * i + n];
    for (int k = 0; k < 4; ++k) f[4 + 4 * n + k] = sg * hist(a, j, r, b1 - k);
  }
  f[20] = a.b[i * a.R + r] * a.inv_diag[i];
  for (int n = 0; n < 4; ++n) {
    const int64_t j = a.nb[4 * i + n];
    f[21 + n] = (double)a.nbs[4 * i + n] * a.b[j * a.R + r] * a.inv_diag[j];
  }
  double ss = 0.0;
  for (int k = 0; k < kF; ++k) ss += f[k] * f[k];
  s = sqrt(ss / kF);
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  for (int k = 0; k < kF; ++k) x[k] = (float)(f[k] * inv);
  xc = 4.0 * f[0] - 6.0 * f[1] + 4.0 * f[2] - f[3];
}

// y = w3 . tanh(W2 tanh(W1 x)) with the parameters in shared memory
__device__ __forceinline__ float mlp_forward(const float* W, const float* x) {
  const float* W1 = W;
  const float* W2 = W + kH * kF;
  const float* w3 = W + kH * kF + kH * kH;
  float h1[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float z = 0.f;
#pragma unroll
    for (int f = 0; f < kF; ++f) z += W1[j * kF + f] * x[f];
    h1[j] = tanhf(z);
  }
  float y = 0.f;
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float z = 0.f;
#pragma unroll
    for (int k = 0; k < kH; ++k) z += W2[j * kH + k] * h1[k];
    y += w3[j] * tanhf(z);
  }
  return y;
}

__device__ __forceinline__ void load_params(const float* Wg, float* Ws) {
  for (int k = threadIdx.x; k < kNP; k += blockDim.x) Ws[k] = Wg[k];
  __syncthreads();
}

// x0[i*R + r] = xc + s y(f/s) for every (edge, RHS)
__global__ void __launch_bounds__(128) k_mlp_infer(FeatArgs a, const float* Wg, double* x0) {
  __shared__ float Ws[kNP];
  load_params(Wg, Ws);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.ne * a.R) return;
  const int64_t i = t / a.R;
  const int r = (int)(t - i * a.R);
  float x[kF];
  double s, xc;
  features(a, i, r, x, s, xc);
  x0[t] = s > 0.0 ? xc + s * (double)mlp_forward(Ws, x) : xc;
}

// y for caller rows X [n][kF]
__global__ void __launch_bounds__(128) k_mlp_forward_rows(const float* X, int64_t n, const float* Wg, float* Y) {
  __shared__ float Ws[kNP];
  load_params(Wg, Ws);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  float x[kF];
  for (int f = 0; f < kF; ++f) x[f] = X[t * kF + f];
  Y[t] = mlp_forward(Ws, x);
}

// training sample of (edge, RHS) for the step just solved: x = f / s,
// t = (J^{alpha-1} - xc) / s (zeros where s = 0) and the raw weight s^2
__global__ void k_mlp_record(FeatArgs a, const double* J, int64_t base, float* X, float* T, float* Wt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.ne * a.R) return;
  const int64_t i = t / a.R;
  const int r = (int)(t - i * a.R);
  float x[kF];
  double s, xc;
  features(a, i, r, x, s, xc);
  float* xo = X + (base + t) * kF;
  for (int f = 0; f < kF; ++f) xo[f] = x[f];
  T[base + t] = s > 0.0 ? (float)((J[t] - xc) / s) : 0.f;
  Wt[base + t] = (float)(s * s);
}

// Weights of one step's samples: s^2 divided by the step's mean of s^2 t^2.
// The weighted loss w (y - t)^2 of a step then is the squared error of the
// guess divided by that of the plain extrapolation (1 for y = 0): each step
// counts by how much the network improves on the extrapolation there, which
// is what the solve's fallback compares.  A step whose extrapolation is exact
// gets weight zero.
__global__ void k_mlp_weight_norm(float* Wt, const float* T, int64_t n) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc += (double)Wt[k] * (double)T[k] * (double)T[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    red[0] = t;
  }
  __syncthreads();
  const double mean = red[0] / (double)n;
  const float sc = mean > 0.0 ? (float)(1.0 / mean) : 0.f;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) Wt[k] *= sc;
}

// One minibatch: samples perm[b0 + k] for k < nb (nb <= gridDim.x * kTB).
// Loss (1/nb) sum w (y - t)^2 (w = 1 when Wt is null) is added to *loss;
// gradients are added to G.
__global__ void __launch_bounds__(kTB) k_mlp_train(const float* X, const float* T, const float* Wt,
                                                   const int32_t* perm, int64_t b0, int32_t nb, const float* Wg,
                                                   float* G, double* loss) {
  extern __shared__ float sm[];
  float* Ws = sm;                    // kNP
  float* xs = Ws + kNP;              // [kTB][kF]
  float* h1s = xs + kTB * kF;        // [kTB][kHS]
  float* h2s = h1s + kTB * kHS;      // [kTB][kHS]
  float* d1s = h2s + kTB * kHS;      // dL/dz1 [kTB][kHS]
  float* d2s = d1s + kTB * kHS;      // dL/dz2 [kTB][kHS]
  float* dys = d2s + kTB * kHS;      // dL/dy [kTB]
  __shared__ double lsum[kTB / 32];
  load_params(Wg, Ws);
  const float* W1 = Ws;
  const float* W2 = Ws + kH * kF;
  const float* w3 = Ws + kH * kF + kH * kH;
  const int s = threadIdx.x;
  const int k = blockIdx.x * kTB + s;
  const bool valid = k < nb;
  const int64_t idx = valid ? (int64_t)(perm ? perm[b0 + k] : b0 + k) : 0;
  float* x = xs + s * kF;
  for (int f = 0; f < kF; ++f) x[f] = valid ? X[idx * kF + f] : 0.f;
  // forward
  float* h1 = h1s + s * kHS;
  float* h2 = h2s + s * kHS;
  for (int j = 0; j < kH; ++j) {
    float z = 0.f;
    for (int f = 0; f < kF; ++f) z += W1[j * kF + f] * x[f];
    h1[j] = tanhf(z);
  }
  float y = 0.f;
  for (int j = 0; j < kH; ++j) {
    float z = 0.f;
    for (int q = 0; q < kH; ++q) z += W2[j * kH + q] * h1[q];
    h2[j] = tanhf(z);
    y += w3[j] * h2[j];
  }
  const float e = valid ? y - T[idx] : 0.f;
  const float wt = valid ? (Wt ? Wt[idx] : 1.f) : 0.f;
  const float dy = 2.f * wt * e / (float)nb;
  dys[s] = dy;
  // backward through the two hidden layers
  float* d2 = d2s + s * kHS;
  float* d1 = d1s + s * kHS;
  for (int j = 0; j < kH; ++j) d2[j] = dy * w3[j] * (1.f - h2[j] * h2[j]);
  for (int q = 0; q < kH; ++q) {
    float acc = 0.f;
    for (int j = 0; j < kH; ++j) acc += d2[j] * W2[j * kH + q];
    d1[q] = acc * (1.f - h1[q] * h1[q]);
  }
  // loss
  double l = valid ? (double)wt * (double)e * (double)e / (double)nb : 0.0;
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((s & 31) == 0) lsum[s >> 5] = l;
  __syncthreads();
  if (s == 0) {
    double t = 0.0;
    for (int w = 0; w < kTB / 32; ++w) t += lsum[w];
    atomicAdd(loss, t);
  }
  // parameter gradients: sums over this block's samples
  for (int o = s; o < kNP; o += kTB) {
    float g = 0.f;
    if (o < kH * kF) {
      const int j = o / kF, f = o - j * kF;
      for (int q = 0; q < kTB; ++q) g += d1s[q * kHS + j] * xs[q * kF + f];
    } else if (o < kH * kF + kH * kH) {
      const int oo = o - kH * kF, j = oo / kH, c = oo - j * kH;
      for (int q = 0; q < kTB; ++q) g += d2s[q * kHS + j] * h1s[q * kHS + c];
    } else {
      const int j = o - kH * kF - kH * kH;
      for (int q = 0; q < kTB; ++q) g += dys[q] * h2s[q * kHS + j];
    }
    atomicAdd(&G[o], g);
  }
}

__global__ void k_mlp_adam(float* W, float* G, float* M, float* V, int n, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float g = G[k];
  const float m = b1 * M[k] + (1.f - b1) * g;
  const float v = b2 * V[k] + (1.f - b2) * g * g;
  M[k] = m;
  V[k] = v;
  W[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  G[k] = 0.f;
}

constexpr size_t kTrainSmem =
    sizeof(float) * ((size_t)kNP + (size_t)kTB * kF + 4 * (size_t)kTB * kHS + (size_t)kTB);

}  // namespace tdbem

using namespace tdbem;

struct Mlp {
  float* w = nullptr;   // parameters [kNP]
  float* g = nullptr;   // gradient accumulator
  float* m = nullptr;   // Adam moments
  float* v = nullptr;
  int64_t adam_t = 0;
  int32_t* nb = nullptr;   // [ne][4]
  int8_t* nbs = nullptr;   // [ne][4]
  float* X = nullptr;      // training samples [cap][kF]
  float* T = nullptr;      // [cap]
  float* Wt = nullptr;     // [cap] sample weights
  int64_t cap = 0, count = 0;
  bool use = false;
  bool have_w = false;     // parameters set by the caller
  double* loss = nullptr;  // device accumulator
  int32_t* perm = nullptr; // [cap]
};

static void mlp_free_buffers(Mlp* M) {
  for (void* p : {(void*)M->w, (void*)M->g, (void*)M->m, (void*)M->v, (void*)M->nb, (void*)M->nbs, (void*)M->X,
                  (void*)M->T, (void*)M->Wt, (void*)M->loss, (void*)M->perm})
    if (p) cudaFree(p);
}

void tdbem_mlp_free(tdbem_ctx* c) {
  if (!c->mlp) return;
  mlp_free_buffers(c->mlp);
  delete c->mlp;
  c->mlp = nullptr;
}

#define MLP_TRY(call)                                                             \
  do {                                                                            \
    cudaError_t e__ = (call);                                                     \
    if (e__ != cudaSuccess) {                                                     \
      c->set_error(std::string("mlp: ") + #call + ": " + cudaGetErrorString(e__)); \
      return e__ == cudaErrorMemoryAllocation ? TDBEM_ENOMEM : TDBEM_ECUDA;       \
    }                                                                             \
  } while (0)

// Network state and the neighbour table (other two sides of the + and the -
// triangle of every edge, signs relative to the edge).
static tdbem_status mlp_init(tdbem_ctx* c) {
  if (c->mlp) return TDBEM_OK;
  Mlp* M = new (std::nothrow) Mlp();
  if (!M) return TDBEM_ENOMEM;
  c->mlp = M;
  MLP_TRY(cudaMalloc(&M->w, kNP * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->g, kNP * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->m, kNP * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->v, kNP * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->loss, sizeof(double)));
  MLP_TRY(cudaMalloc(&M->nb, 4 * c->ne * sizeof(int32_t)));
  MLP_TRY(cudaMalloc(&M->nbs, 4 * c->ne * sizeof(int8_t)));
  std::vector<int32_t> nb(4 * c->ne);
  std::vector<int8_t> nbs(4 * c->ne);
  for (int64_t i = 0; i < c->ne; ++i) {
    for (int rho = 0; rho < 2; ++rho) {
      const int32_t t = c->et[2 * i + rho];
      int k = 0;
      while (k < 3 && c->te[3 * t + k] != i) ++k;
      if (k == 3) {
        c->set_error("mlp: edge table inconsistent");
        return TDBEM_EMESH;
      }
      for (int u = 1; u <= 2; ++u) {
        const int kk = (k + u) % 3;
        nb[4 * i + 2 * rho + (u - 1)] = c->te[3 * t + kk];
        nbs[4 * i + 2 * rho + (u - 1)] = (int8_t)(c->ts[3 * t + k] * c->ts[3 * t + kk]);
      }
    }
  }
  MLP_TRY(cudaMemcpy(M->nb, nb.data(), nb.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  MLP_TRY(cudaMemcpy(M->nbs, nbs.data(), nbs.size() * sizeof(int8_t), cudaMemcpyHostToDevice));
  MLP_TRY(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem));
  return TDBEM_OK;
}

static FeatArgs feat_args(tdbem_ctx* c, int32_t alpha) {
  FeatArgs a;
  a.ring = c->d_Jring;
  a.b = c->d_R;
  a.inv_diag = c->d_z0_inv_diag;
  a.nb = c->mlp->nb;
  a.nbs = c->mlp->nbs;
  a.ne = c->ne;
  a.L = c->L;
  a.R = c->R;
  a.alpha = alpha;
  return a;
}

// Before the solve of step alpha: the network's guess into d_J (warm = 2).
tdbem_status tdbem_mlp_before_solve(tdbem_ctx* c, int32_t alpha, int32_t* warm) {
  if (!c->mlp || !c->mlp->use) return TDBEM_OK;
  const int64_t n = c->ne * (int64_t)c->R;
  k_mlp_infer<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(feat_args(c, alpha), c->mlp->w, c->d_J);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  *warm = 2;
  return TDBEM_OK;
}

// After the solve of step alpha: record its samples while there is room.
tdbem_status tdbem_mlp_after_solve(tdbem_ctx* c, int32_t alpha) {
  Mlp* M = c->mlp;
  if (!M || !M->X) return TDBEM_OK;
  const int64_t n = c->ne * (int64_t)c->R;
  if (M->count + n > M->cap) return TDBEM_OK;
  k_mlp_record<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(feat_args(c, alpha), c->d_J, M->count, M->X,
                                                                   M->T, M->Wt);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  k_mlp_weight_norm<<<1, 1024, 0, c->stream>>>(M->Wt + M->count, M->T + M->count, n);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  M->count += n;
  return TDBEM_OK;
}

// splitmix64 (Steele, Lea and Flood, 2014) for the per-epoch shuffles
static uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" {

tdbem_status tdbem_mlp_set_weights(tdbem_ctx* c, const float* theta) {
  if (!c || !theta) return TDBEM_EINVAL;
  tdbem_status s = mlp_init(c);
  if (s) return s;
  Mlp* M = c->mlp;
  MLP_TRY(cudaMemcpyAsync(M->w, theta, kNP * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  MLP_TRY(cudaMemsetAsync(M->g, 0, kNP * sizeof(float), c->stream));
  MLP_TRY(cudaMemsetAsync(M->m, 0, kNP * sizeof(float), c->stream));
  MLP_TRY(cudaMemsetAsync(M->v, 0, kNP * sizeof(float), c->stream));
  MLP_TRY(cudaStreamSynchronize(c->stream));
  M->adam_t = 0;
  M->have_w = true;
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_get_weights(tdbem_ctx* c, float* theta) {
  if (!c || !theta) return TDBEM_EINVAL;
  if (!c->mlp || !c->mlp->have_w) {
    c->set_error("mlp: no weights set");
    return TDBEM_ESTATE;
  }
  MLP_TRY(cudaMemcpyAsync(theta, c->mlp->w, kNP * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaStreamSynchronize(c->stream));
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_record(tdbem_ctx* c, int64_t capacity) {
  if (!c || capacity < 0) return TDBEM_EINVAL;
  tdbem_status s = mlp_init(c);
  if (s) return s;
  Mlp* M = c->mlp;
  MLP_TRY(cudaStreamSynchronize(c->stream));
  for (void* p : {(void*)M->X, (void*)M->T, (void*)M->Wt, (void*)M->perm})
    if (p) cudaFree(p);
  M->X = nullptr;
  M->T = nullptr;
  M->Wt = nullptr;
  M->perm = nullptr;
  M->cap = M->count = 0;
  if (capacity == 0) return TDBEM_OK;
  MLP_TRY(cudaMalloc(&M->X, capacity * kF * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->T, capacity * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->Wt, capacity * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->perm, capacity * sizeof(int32_t)));
  M->cap = capacity;
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_samples(tdbem_ctx* c, int64_t first, int64_t n, float* X, float* T, float* Wt,
                               int64_t* count) {
  if (!c || first < 0 || n < 0) return TDBEM_EINVAL;
  Mlp* M = c->mlp;
  if (count) *count = M ? M->count : 0;
  if (n == 0) return TDBEM_OK;
  if (!M || first + n > M->count) return TDBEM_EINVAL;
  if (X) MLP_TRY(cudaMemcpyAsync(X, M->X + first * kF, n * kF * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (T) MLP_TRY(cudaMemcpyAsync(T, M->T + first, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (Wt) MLP_TRY(cudaMemcpyAsync(Wt, M->Wt + first, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaStreamSynchronize(c->stream));
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_train(tdbem_ctx* c, int32_t epochs, int32_t batch, float lr, uint64_t seed, float* loss) {
  if (!c || epochs < 0 || batch < kTB || batch % kTB || !(lr > 0)) return TDBEM_EINVAL;
  Mlp* M = c->mlp;
  if (!M || !M->X || M->count == 0 || !M->have_w) {
    c->set_error("mlp: no recorded samples or no weights set");
    return TDBEM_ESTATE;
  }
  if (M->count > INT32_MAX) return TDBEM_EINVAL;
  const int64_t n = M->count;
  std::vector<int32_t> perm(n);
  uint64_t st = seed;
  for (int32_t ep = 0; ep < epochs; ++ep) {
    for (int64_t k = 0; k < n; ++k) perm[k] = (int32_t)k;
    for (int64_t k = n - 1; k > 0; --k) {  // Fisher-Yates
      const int64_t j = (int64_t)(splitmix64(st) % (uint64_t)(k + 1));
      std::swap(perm[k], perm[j]);
    }
    MLP_TRY(cudaMemcpyAsync(M->perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    MLP_TRY(cudaMemsetAsync(M->loss, 0, sizeof(double), c->stream));
    int64_t nbatch = 0;
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int32_t nb = (int32_t)std::min<int64_t>(batch, n - b0);
      k_mlp_train<<<(unsigned)((nb + kTB - 1) / kTB), kTB, kTrainSmem, c->stream>>>(M->X, M->T, M->Wt, M->perm, b0,
                                                                                       nb, M->w, M->g, M->loss);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
      ++M->adam_t;
      const float c1 = 1.f - powf(0.9f, (float)M->adam_t), c2 = 1.f - powf(0.999f, (float)M->adam_t);
      k_mlp_adam<<<(kNP + 255) / 256, 256, 0, c->stream>>>(M->w, M->g, M->m, M->v, kNP, lr, 0.9f, 0.999f, 1e-8f, c1,
                                                           c2);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
      ++nbatch;
    }
    double l = 0.0;
    MLP_TRY(cudaMemcpyAsync(&l, M->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MLP_TRY(cudaStreamSynchronize(c->stream));
    if (loss) loss[ep] = (float)(l / (double)nbatch);
  }
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_grad(tdbem_ctx* c, const float* X, const float* T, const float* Wt, int64_t n, float* loss,
                            float* grad) {
  if (!c || !X || !T || n < 1 || n > INT32_MAX || !grad) return TDBEM_EINVAL;
  Mlp* M = c->mlp;
  if (!M || !M->have_w) {
    c->set_error("mlp: no weights set");
    return TDBEM_ESTATE;
  }
  float *dX = nullptr, *dT = nullptr, *dW = nullptr;
  MLP_TRY(cudaMallocAsync(&dX, n * kF * sizeof(float), c->stream));
  MLP_TRY(cudaMallocAsync(&dT, n * sizeof(float), c->stream));
  MLP_TRY(cudaMemcpyAsync(dX, X, n * kF * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  MLP_TRY(cudaMemcpyAsync(dT, T, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  if (Wt) {
    MLP_TRY(cudaMallocAsync(&dW, n * sizeof(float), c->stream));
    MLP_TRY(cudaMemcpyAsync(dW, Wt, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  }
  MLP_TRY(cudaMemsetAsync(M->g, 0, kNP * sizeof(float), c->stream));
  MLP_TRY(cudaMemsetAsync(M->loss, 0, sizeof(double), c->stream));
  k_mlp_train<<<(unsigned)((n + kTB - 1) / kTB), kTB, kTrainSmem, c->stream>>>(dX, dT, dW, nullptr, 0, (int32_t)n,
                                                                                M->w, M->g, M->loss);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  double l = 0.0;
  MLP_TRY(cudaMemcpyAsync(grad, M->g, kNP * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaMemcpyAsync(&l, M->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaMemsetAsync(M->g, 0, kNP * sizeof(float), c->stream));
  cudaFreeAsync(dX, c->stream);
  cudaFreeAsync(dT, c->stream);
  if (dW) cudaFreeAsync(dW, c->stream);
  MLP_TRY(cudaStreamSynchronize(c->stream));
  if (loss) *loss = (float)l;
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_forward(tdbem_ctx* c, const float* X, int64_t n, float* Y) {
  if (!c || !X || !Y || n < 1) return TDBEM_EINVAL;
  Mlp* M = c->mlp;
  if (!M || !M->have_w) {
    c->set_error("mlp: no weights set");
    return TDBEM_ESTATE;
  }
  float *dX = nullptr, *dY = nullptr;
  MLP_TRY(cudaMallocAsync(&dX, n * kF * sizeof(float), c->stream));
  MLP_TRY(cudaMallocAsync(&dY, n * sizeof(float), c->stream));
  MLP_TRY(cudaMemcpyAsync(dX, X, n * kF * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  k_mlp_forward_rows<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(dX, n, M->w, dY);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  MLP_TRY(cudaMemcpyAsync(Y, dY, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  cudaFreeAsync(dX, c->stream);
  cudaFreeAsync(dY, c->stream);
  MLP_TRY(cudaStreamSynchronize(c->stream));
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_use(tdbem_ctx* c, int32_t on) {
  if (!c) return TDBEM_EINVAL;
  if (on && (!c->mlp || !c->mlp->have_w)) {
    c->set_error("mlp: no weights set");
    return TDBEM_ESTATE;
  }
  if (c->mlp) c->mlp->use = on != 0;
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_stats(tdbem_ctx* c, int64_t* used, int64_t* fallback) {
  if (!c) return TDBEM_EINVAL;
  int32_t h[2] = {0, 0};
  MLP_TRY(cudaMemcpyAsync(h, c->d_status + 8, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaStreamSynchronize(c->stream));
  if (used) *used = h[0];
  if (fallback) *fallback = h[1];
  return TDBEM_OK;
}

}  // extern "C"
