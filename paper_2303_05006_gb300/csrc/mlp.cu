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
//
// Width 256 (tdbem_mlp_set_width) runs the two dense layers and the weight
// gradients as products on the tcgen05 tensor cores (gemm_tc.cu: BF16
// operands, FP32 accumulation; FP32 master parameters, FP32 Adam).  A pass
// over n rows is: features or gathered samples -> X (BF16, 25 features padded
// to 32) -> Z1 = X W1^T -> H1 = tanh Z1 -> Z2 = H1 W2^T -> head (y, and for
// training the loss, dy and D2 = dy w3 (1 - h2^2)); training then forms
// dW2 = D2^T H1, dH1 = D2 W2, D1 = dH1 (1 - h1^2) and dW1 = D1^T X, the
// products over the batch taking the transposed BF16 copies as K-major
// operands (k_bf16_transpose).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include <cuda_bf16.h>

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

// ---- width 256 on the tensor cores ----
constexpr int kH2 = 256, kFP = 32;  // width; features padded to 32 (the products' K is a multiple of 8)
constexpr int64_t kNP2 = (int64_t)kH2 * kF + (int64_t)kH2 * kH2 + kH2;

// FP32 master parameters -> BF16 operands: W1 [H][F] -> wb1 [H][32]
// (zero-padded), W2 [H][H] -> wb2 and its transpose wb2t
__global__ void k_mlp_cast(const float* W, __nv_bfloat16* wb1, __nv_bfloat16* wb2, __nv_bfloat16* wb2t) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kH2 * kFP) {
    const int j = t / kFP, f = t - j * kFP;
    wb1[t] = __float2bfloat16_rn(f < kF ? W[j * kF + f] : 0.f);
  }
  if (t < kH2 * kH2) {
    const int j = t / kH2, k = t - j * kH2;
    const __nv_bfloat16 v = __float2bfloat16_rn(W[kH2 * kF + t]);
    wb2[t] = v;
    wb2t[k * kH2 + j] = v;
  }
}

// inference features of every (edge, RHS) as BF16 rows of 32, with the
// scale and the cubic extrapolation
__global__ void __launch_bounds__(128) k_mlp_feat_tc(FeatArgs a, __nv_bfloat16* xb, double* sx, double* xcx) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.ne * a.R) return;
  const int64_t i = t / a.R;
  const int r = (int)(t - i * a.R);
  float x[kF];
  double s, xc;
  features(a, i, r, x, s, xc);
  for (int f = 0; f < kFP; ++f) xb[t * kFP + f] = __float2bfloat16_rn(f < kF ? x[f] : 0.f);
  sx[t] = s;
  xcx[t] = xc;
}

// rows [b0, b0 + nrows) of a batch: sample perm[b0 + k] (k when perm is null)
// of X as a BF16 row of 32, its target and weight (1 when Wt is null); rows
// k >= nb are zero with zero weight
__global__ void k_mlp_gather_tc(const float* X, const float* T, const float* Wt, const int32_t* perm, int64_t b0,
                                int nb, int nrows, __nv_bfloat16* xb, float* tb, float* wtb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrows * kFP) return;
  const int k = (int)(t / kFP), f = (int)(t - (int64_t)k * kFP);
  const bool v = k < nb;
  const int64_t idx = v ? (int64_t)(perm ? perm[b0 + k] : b0 + k) : 0;
  xb[t] = __float2bfloat16_rn(v && f < kF ? X[idx * kF + f] : 0.f);
  if (f == 0 && tb) {
    tb[k] = v ? T[idx] : 0.f;
    wtb[k] = v ? (Wt ? Wt[idx] : 1.f) : 0.f;
  }
}

// out[c * ldo + r] = in[r * cols + c] (BF16), 32 x 32 tiles through shared memory
__global__ void k_bf16_transpose(const __nv_bfloat16* in, int rows, int cols, __nv_bfloat16* out, int64_t ldo) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(int64_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(int64_t)c * ldo + r] = tile[threadIdx.x][k];
  }
}

__global__ void k_tanh_bf16(const float* z, int64_t n, __nv_bfloat16* h) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) h[t] = __float2bfloat16_rn(tanhf(z[t]));
}

// d1 = dh1 (1 - h1^2) as BF16
__global__ void k_mlp_dtanh(const float* dh1, const __nv_bfloat16* h1b, int64_t n, __nv_bfloat16* d1b) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float h = __bfloat162float(h1b[t]);
  d1b[t] = __float2bfloat16_rn(dh1[t] * (1.f - h * h));
}

// inference head, one warp per row: y = w3 . tanh(z2); x0 = xc + s y (or y
// itself into yout)
__global__ void k_mlp_out_tc(const float* z2, const float* w3, int64_t n, const double* sx, const double* xcx,
                             double* x0, float* yout) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float y = 0.f;
  for (int j = lane; j < kH2; j += 32) y += w3[j] * tanhf(z2[row * kH2 + j]);
  for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
  if (lane == 0) {
    if (yout) yout[row] = y;
    if (x0) x0[row] = sx[row] > 0.0 ? xcx[row] + sx[row] * (double)y : xcx[row];
  }
}

// training head: warps stride over the rows; per row h2 = tanh(z2), y, the
// weighted error, dy = 2 w e / nb, d2 = dy w3 (1 - h2^2) (BF16 into d2b) and
// the loss; dL/dw3 = sum over rows of dy h2, per lane then per block, added
// to g3 once per block
__global__ void __launch_bounds__(256) k_mlp_head_tc(const float* z2, const float* w3, const float* tb,
                                                     const float* wtb, int nrows, int nb, __nv_bfloat16* d2b,
                                                     float* g3, double* loss) {
  __shared__ float g3s[kH2];
  __shared__ double ls[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = threadIdx.x; j < kH2; j += blockDim.x) g3s[j] = 0.f;
  __syncthreads();
  float g[kH2 / 32];
#pragma unroll
  for (int q = 0; q < kH2 / 32; ++q) g[q] = 0.f;
  double lw = 0.0;
  for (int row = blockIdx.x * 8 + warp; row < nrows; row += gridDim.x * 8) {
    float h2[kH2 / 32];
    float y = 0.f;
#pragma unroll
    for (int q = 0; q < kH2 / 32; ++q) {
      h2[q] = tanhf(z2[(int64_t)row * kH2 + lane + 32 * q]);
      y += w3[lane + 32 * q] * h2[q];
    }
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    const float e = y - tb[row], w = wtb[row];
    const float dy = 2.f * w * e / (float)nb;
    lw += (double)w * (double)e * (double)e / (double)nb;
#pragma unroll
    for (int q = 0; q < kH2 / 32; ++q) {
      const int j = lane + 32 * q;
      d2b[(int64_t)row * kH2 + j] = __float2bfloat16_rn(dy * w3[j] * (1.f - h2[q] * h2[q]));
      g[q] += dy * h2[q];
    }
  }
#pragma unroll
  for (int q = 0; q < kH2 / 32; ++q) atomicAdd(&g3s[lane + 32 * q], g[q]);
  if (lane == 0) ls[warp] = lw;  // lw is the same in every lane
  __syncthreads();
  for (int j = threadIdx.x; j < kH2; j += blockDim.x) atomicAdd(&g3[j], g3s[j]);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ls[w];
    atomicAdd(loss, t);
  }
}

// G1 [H][F] += g1p[:, :F] (g1p [H][32])
__global__ void k_mlp_fold_g1(const float* g1p, float* G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kH2 * kF) return;
  const int j = t / kF, f = t - j * kF;
  G[t] += g1p[j * kFP + f];
}

constexpr size_t kTrainSmem =
    sizeof(float) * ((size_t)kNP + (size_t)kTB * kF + 4 * (size_t)kTB * kHS + (size_t)kTB);

}  // namespace tdbem

using namespace tdbem;

struct Mlp {
  int H = kH;           // width: 64 (FP32 CUDA cores) or 256 (tensor cores)
  int64_t np = kNP;     // parameters of that width
  float* w = nullptr;   // parameters [np]
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
  int32_t every = 1;       // record the steps alpha with alpha % every == 0
  bool use = false;
  bool have_w = false;     // parameters set by the caller
  double* loss = nullptr;  // device accumulator
  int32_t* perm = nullptr; // [cap]
  // width 256: BF16 operand copies of the parameters and the work rows
  __nv_bfloat16 *wb1 = nullptr, *wb2 = nullptr, *wb2t = nullptr;
  int64_t rows_cap = 0;
  __nv_bfloat16 *xb = nullptr, *xbt = nullptr, *h1b = nullptr, *h1bt = nullptr, *d2b = nullptr, *d2bt = nullptr,
                *d1b = nullptr, *d1bt = nullptr;
  float *z = nullptr, *tb = nullptr, *wtb = nullptr, *g1p = nullptr;
  double *sx = nullptr, *xcx = nullptr;
  int32_t* err = nullptr;
};

static void mlp_free_rows(Mlp* M) {
  for (void* p : {(void*)M->xb, (void*)M->xbt, (void*)M->h1b, (void*)M->h1bt, (void*)M->d2b, (void*)M->d2bt,
                  (void*)M->d1b, (void*)M->d1bt, (void*)M->z, (void*)M->tb, (void*)M->wtb, (void*)M->sx,
                  (void*)M->xcx})
    if (p) cudaFree(p);
  M->xb = M->xbt = M->h1b = M->h1bt = M->d2b = M->d2bt = M->d1b = M->d1bt = nullptr;
  M->z = M->tb = M->wtb = nullptr;
  M->sx = M->xcx = nullptr;
  M->rows_cap = 0;
}

static void mlp_free_params(Mlp* M) {
  for (void* p : {(void*)M->w, (void*)M->g, (void*)M->m, (void*)M->v, (void*)M->wb1, (void*)M->wb2, (void*)M->wb2t,
                  (void*)M->g1p})
    if (p) cudaFree(p);
  M->w = M->g = M->m = M->v = M->g1p = nullptr;
  M->wb1 = M->wb2 = M->wb2t = nullptr;
}

static void mlp_free_buffers(Mlp* M) {
  mlp_free_params(M);
  mlp_free_rows(M);
  for (void* p : {(void*)M->nb, (void*)M->nbs, (void*)M->X, (void*)M->T, (void*)M->Wt, (void*)M->loss,
                  (void*)M->perm, (void*)M->err})
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
  MLP_TRY(cudaMalloc(&M->loss, sizeof(double)));
  MLP_TRY(cudaMalloc(&M->err, sizeof(int32_t)));
  MLP_TRY(cudaMemset(M->err, 0, sizeof(int32_t)));
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

// Parameter buffers of the current width (and, for width 256, the BF16
// operand copies and the padded first-layer gradient).
static tdbem_status mlp_alloc_params(tdbem_ctx* c) {
  Mlp* M = c->mlp;
  if (M->w) return TDBEM_OK;
  MLP_TRY(cudaMalloc(&M->w, M->np * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->g, M->np * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->m, M->np * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->v, M->np * sizeof(float)));
  if (M->H == kH2) {
    MLP_TRY(cudaMalloc(&M->wb1, (size_t)kH2 * kFP * sizeof(__nv_bfloat16)));
    MLP_TRY(cudaMalloc(&M->wb2, (size_t)kH2 * kH2 * sizeof(__nv_bfloat16)));
    MLP_TRY(cudaMalloc(&M->wb2t, (size_t)kH2 * kH2 * sizeof(__nv_bfloat16)));
    MLP_TRY(cudaMalloc(&M->g1p, (size_t)kH2 * kFP * sizeof(float)));
  }
  return TDBEM_OK;
}

// Work rows of the width-256 passes, grown to hold n rows (a multiple of 128).
static tdbem_status mlp_rows(tdbem_ctx* c, int64_t n) {
  Mlp* M = c->mlp;
  if (n <= M->rows_cap) return TDBEM_OK;
  MLP_TRY(cudaStreamSynchronize(c->stream));
  mlp_free_rows(M);
  const size_t hb = (size_t)n * kH2 * sizeof(__nv_bfloat16), xbsz = (size_t)n * kFP * sizeof(__nv_bfloat16);
  MLP_TRY(cudaMalloc(&M->xb, xbsz));
  MLP_TRY(cudaMalloc(&M->xbt, xbsz));
  for (__nv_bfloat16** p : {&M->h1b, &M->h1bt, &M->d2b, &M->d2bt, &M->d1b, &M->d1bt}) MLP_TRY(cudaMalloc(p, hb));
  MLP_TRY(cudaMalloc(&M->z, (size_t)n * kH2 * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->tb, n * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->wtb, n * sizeof(float)));
  MLP_TRY(cudaMalloc(&M->sx, n * sizeof(double)));
  MLP_TRY(cudaMalloc(&M->xcx, n * sizeof(double)));
  M->rows_cap = n;
  return TDBEM_OK;
}

// BF16 operand copies of the current parameters (width 256)
static tdbem_status mlp_cast(tdbem_ctx* c) {
  Mlp* M = c->mlp;
  k_mlp_cast<<<(kH2 * kH2 + 255) / 256, 256, 0, c->stream>>>(M->w, M->wb1, M->wb2, M->wb2t);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

static tdbem_status mlp_check_err(tdbem_ctx* c) {
  int32_t e = 0;
  MLP_TRY(cudaMemcpyAsync(&e, c->mlp->err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaStreamSynchronize(c->stream));
  if (e) {
    c->set_error("mlp: a tensor-core product timed out");
    return TDBEM_ETIMEOUT;
  }
  return TDBEM_OK;
}

// Width 256: the two dense layers over rows xb [n] (n a multiple of 128) ->
// z = Z2 and h1b = tanh(Z1)
static tdbem_status mlp_forward_tc(tdbem_ctx* c, int64_t n) {
  Mlp* M = c->mlp;
  tdbem_status s;
  if ((s = tdbem_gemm_bf16(c, c->stream, M->xb, kFP, M->wb1, kFP, M->z, kH2, (int)n, kH2, kFP, 0, 1, M->err)))
    return s;
  k_tanh_bf16<<<(unsigned)((n * kH2 + 255) / 256), 256, 0, c->stream>>>(M->z, n * kH2, M->h1b);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return tdbem_gemm_bf16(c, c->stream, M->h1b, kH2, M->wb2, kH2, M->z, kH2, (int)n, kH2, kH2, 0, 1, M->err);
}

// Width 256, one batch of nrows gathered rows (nb of them real): loss into
// M->loss, gradient added to M->g
static tdbem_status mlp_backward_tc(tdbem_ctx* c, int nrows, int nb) {
  Mlp* M = c->mlp;
  tdbem_status s;
  if ((s = mlp_forward_tc(c, nrows))) return s;
  float* G1 = M->g;
  float* G2 = M->g + (int64_t)kH2 * kF;
  float* G3 = G2 + (int64_t)kH2 * kH2;
  k_mlp_head_tc<<<std::max(1, std::min(nrows / 8, 304)), 256, 0, c->stream>>>(M->z, M->w + kH2 * kF + kH2 * kH2,
                                                                              M->tb, M->wtb, nrows, nb, M->d2b, G3,
                                                                              M->loss);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  const dim3 tb(32, 8);
  k_bf16_transpose<<<dim3(kH2 / 32, nrows / 32), tb, 0, c->stream>>>(M->d2b, nrows, kH2, M->d2bt, nrows);
  k_bf16_transpose<<<dim3(kH2 / 32, nrows / 32), tb, 0, c->stream>>>(M->h1b, nrows, kH2, M->h1bt, nrows);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  const int ksplit = std::max(1, nrows / 256);  // two 128-row tiles of dW2: about nrows / 128 CTAs
  // dW2 = D2^T H1
  if ((s = tdbem_gemm_bf16(c, c->stream, M->d2bt, nrows, M->h1bt, nrows, G2, kH2, kH2, kH2, nrows, 1, ksplit,
                           M->err)))
    return s;
  // dH1 = D2 W2 (into z), D1 = dH1 (1 - h1^2)
  if ((s = tdbem_gemm_bf16(c, c->stream, M->d2b, kH2, M->wb2t, kH2, M->z, kH2, nrows, kH2, kH2, 0, 1, M->err)))
    return s;
  k_mlp_dtanh<<<(unsigned)(((int64_t)nrows * kH2 + 255) / 256), 256, 0, c->stream>>>(M->z, M->h1b,
                                                                                     (int64_t)nrows * kH2, M->d1b);
  k_bf16_transpose<<<dim3(kH2 / 32, nrows / 32), tb, 0, c->stream>>>(M->d1b, nrows, kH2, M->d1bt, nrows);
  k_bf16_transpose<<<dim3(kFP / 32, nrows / 32), tb, 0, c->stream>>>(M->xb, nrows, kFP, M->xbt, nrows);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  // dW1 = D1^T X (padded to 32 columns, then folded into G1)
  MLP_TRY(cudaMemsetAsync(M->g1p, 0, (size_t)kH2 * kFP * sizeof(float), c->stream));
  if ((s = tdbem_gemm_bf16(c, c->stream, M->d1bt, nrows, M->xbt, nrows, M->g1p, kFP, kH2, kFP, nrows, 1,
                           std::max(1, nrows / 128), M->err)))
    return s;
  k_mlp_fold_g1<<<(kH2 * kF + 255) / 256, 256, 0, c->stream>>>(M->g1p, G1);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
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
  Mlp* M = c->mlp;
  const int64_t n = c->ne * (int64_t)c->R;
  if (M->H == kH2) {
    const int64_t nr = (n + 127) / 128 * 128;
    tdbem_status s;
    if ((s = mlp_rows(c, nr))) return s;
    if (nr > n) MLP_TRY(cudaMemsetAsync(M->xb + n * kFP, 0, (nr - n) * kFP * sizeof(__nv_bfloat16), c->stream));
    k_mlp_feat_tc<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(feat_args(c, alpha), M->xb, M->sx, M->xcx);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    if ((s = mlp_forward_tc(c, nr))) return s;
    k_mlp_out_tc<<<(unsigned)((n * 32 + 255) / 256), 256, 0, c->stream>>>(M->z, M->w + kH2 * kF + kH2 * kH2, n,
                                                                          M->sx, M->xcx, c->d_J, nullptr);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  } else {
    k_mlp_infer<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(feat_args(c, alpha), M->w, c->d_J);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
  *warm = 2;
  return TDBEM_OK;
}

// After the solve of step alpha: record its samples while there is room.
tdbem_status tdbem_mlp_after_solve(tdbem_ctx* c, int32_t alpha) {
  Mlp* M = c->mlp;
  if (!M || !M->X || alpha % M->every) return TDBEM_OK;
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

tdbem_status tdbem_mlp_set_width(tdbem_ctx* c, int32_t width) {
  if (!c || (width != kH && width != kH2)) return TDBEM_EINVAL;
  tdbem_status s = mlp_init(c);
  if (s) return s;
  Mlp* M = c->mlp;
  MLP_TRY(cudaStreamSynchronize(c->stream));
  mlp_free_params(M);
  mlp_free_rows(M);
  M->H = width;
  M->np = (int64_t)width * kF + (int64_t)width * width + width;
  M->have_w = false;
  M->use = false;
  return TDBEM_OK;
}

tdbem_status tdbem_mlp_set_weights(tdbem_ctx* c, const float* theta) {
  if (!c || !theta) return TDBEM_EINVAL;
  tdbem_status s = mlp_init(c);
  if (s || (s = mlp_alloc_params(c))) return s;
  Mlp* M = c->mlp;
  MLP_TRY(cudaMemcpyAsync(M->w, theta, M->np * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  MLP_TRY(cudaMemsetAsync(M->g, 0, M->np * sizeof(float), c->stream));
  MLP_TRY(cudaMemsetAsync(M->m, 0, M->np * sizeof(float), c->stream));
  MLP_TRY(cudaMemsetAsync(M->v, 0, M->np * sizeof(float), c->stream));
  if (M->H == kH2 && (s = mlp_cast(c))) return s;
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
  MLP_TRY(cudaMemcpyAsync(theta, c->mlp->w, c->mlp->np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
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

tdbem_status tdbem_mlp_record_every(tdbem_ctx* c, int32_t every) {
  if (!c || every < 1) return TDBEM_EINVAL;
  tdbem_status s = mlp_init(c);
  if (s) return s;
  c->mlp->every = every;
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
      if (M->H == kH2) {
        const int nrows = (nb + kTB - 1) / kTB * kTB;
        tdbem_status s;
        if ((s = mlp_rows(c, nrows))) return s;
        k_mlp_gather_tc<<<(unsigned)(((int64_t)nrows * kFP + 255) / 256), 256, 0, c->stream>>>(
            M->X, M->T, M->Wt, M->perm, b0, nb, nrows, M->xb, M->tb, M->wtb);
        TDBEM_CUDA_TRY(c, cudaGetLastError());
        if ((s = mlp_backward_tc(c, nrows, nb))) return s;
      } else {
        k_mlp_train<<<(unsigned)((nb + kTB - 1) / kTB), kTB, kTrainSmem, c->stream>>>(M->X, M->T, M->Wt, M->perm,
                                                                                         b0, nb, M->w, M->g, M->loss);
        TDBEM_CUDA_TRY(c, cudaGetLastError());
      }
      ++M->adam_t;
      const float c1 = 1.f - powf(0.9f, (float)M->adam_t), c2 = 1.f - powf(0.999f, (float)M->adam_t);
      k_mlp_adam<<<(unsigned)((M->np + 255) / 256), 256, 0, c->stream>>>(M->w, M->g, M->m, M->v, (int)M->np, lr,
                                                                          0.9f, 0.999f, 1e-8f, c1, c2);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
      if (M->H == kH2) {
        tdbem_status s;
        if ((s = mlp_cast(c))) return s;
      }
      ++nbatch;
    }
    if (M->H == kH2) {
      tdbem_status s;
      if ((s = mlp_check_err(c))) return s;
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
  MLP_TRY(cudaMemsetAsync(M->g, 0, M->np * sizeof(float), c->stream));
  MLP_TRY(cudaMemsetAsync(M->loss, 0, sizeof(double), c->stream));
  if (M->H == kH2) {
    const int nrows = (int)((n + kTB - 1) / kTB * kTB);
    tdbem_status s;
    if ((s = mlp_rows(c, nrows))) return s;
    k_mlp_gather_tc<<<(unsigned)(((int64_t)nrows * kFP + 255) / 256), 256, 0, c->stream>>>(
        dX, dT, dW, nullptr, 0, (int)n, nrows, M->xb, M->tb, M->wtb);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    if ((s = mlp_backward_tc(c, nrows, (int)n)) || (s = mlp_check_err(c))) return s;
  } else {
    k_mlp_train<<<(unsigned)((n + kTB - 1) / kTB), kTB, kTrainSmem, c->stream>>>(dX, dT, dW, nullptr, 0, (int32_t)n,
                                                                                  M->w, M->g, M->loss);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
  double l = 0.0;
  MLP_TRY(cudaMemcpyAsync(grad, M->g, M->np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaMemcpyAsync(&l, M->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MLP_TRY(cudaMemsetAsync(M->g, 0, M->np * sizeof(float), c->stream));
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
  if (M->H == kH2) {
    const int64_t nrows = (n + kTB - 1) / kTB * kTB;
    tdbem_status s;
    if (nrows > INT32_MAX || (s = mlp_rows(c, nrows))) return nrows > INT32_MAX ? TDBEM_EINVAL : s;
    k_mlp_gather_tc<<<(unsigned)((nrows * kFP + 255) / 256), 256, 0, c->stream>>>(dX, nullptr, nullptr, nullptr, 0,
                                                                                 (int)n, (int)nrows, M->xb, nullptr,
                                                                                 nullptr);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    if ((s = mlp_forward_tc(c, nrows))) return s;
    k_mlp_out_tc<<<(unsigned)((n * 32 + 255) / 256), 256, 0, c->stream>>>(M->z, M->w + kH2 * kF + kH2 * kH2, n,
                                                                          nullptr, nullptr, nullptr, dY);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    if ((s = mlp_check_err(c))) return s;
  } else {
    k_mlp_forward_rows<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(dX, n, M->w, dY);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
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
