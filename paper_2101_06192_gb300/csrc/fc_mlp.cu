// Learned control variate (not in the paper): a two-layer perceptron that
// predicts g_v ~ Omega_vv from local features of v; the prediction only sets
// the control-variate coefficient beta_v = (1 - g_v) / (1 - p_v), so the
// estimator stays unbiased whatever the network outputs.
//
//   features  x = (log(1 + deg), log(1 + alpha d_w), log(1 + sum_{u in N(v)} deg(u)), log(alpha))
//   network   h = relu(W1 x + b1) (128 units), z = w2 . h + b2,
//             g = p + (1 - p) sigmoid(z)
//   loss      mean over vertices of (g - y)^2
//   optimiser Adam (Kingma & Ba) with bias correction
//
// Parameters: one FP32 master vector of MLP_NPARAM floats laid out as
// W1[128][4], b1[128], w2[128], b2.  Every kernel reads them rounded to BF16
// (round to nearest even) and accumulates in FP32.  The hidden layer has K = 4
// and the output layer N = 1, so these are per-vertex dot products on the
// CUDA cores, bound by reading the 16-byte feature rows.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "fc_internal.cuh"

namespace fcx {

constexpr int HID = 128;
constexpr int NF = 4;
constexpr int OFF_W1 = 0, OFF_B1 = HID * NF, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID;
constexpr int NPARAM = OFF_B2 + 1;  // 769
constexpr int MLP_T = 128;          // threads per block (one hidden unit each in the gradient pass)

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ double p_of(const uint4& ri) {
  const uint64_t T = (uint64_t)ri.z | ((uint64_t)ri.w << 32);
  return (double)T * 0x1.0p-53;
}

// Sum over neighbours of their degree, s2[v] = sum over w in N(v) of deg(w).
// A warp takes chunks of NDS_CHUNK consecutive CSR entries and walks each in
// steps of 32: lane i reads entry e0 + i (coalesced column indices), finds its
// row among the 32 row ends that follow the step's first row (a binary search
// over the warp's registers; an entry beyond them, after empty rows, searches
// the row pointers itself), and the lanes of one row add their neighbours'
// degrees with a segmented warp sum whose last lane adds the total to s2 (one
// atomic per row segment, so a hub row is shared by many warps).  The totals
// are integers: any order of the additions gives the same result.
constexpr int NDS_CHUNK = 32 * 32;
constexpr unsigned NDS_FULL = 0xffffffffu;
__device__ __forceinline__ int32_t row_of_entry(const int64_t* __restrict__ rowptr, int32_t lo, int32_t hi,
                                                int64_t e) {
  // the row v in [lo, hi] with rowptr[v] <= e < rowptr[v + 1] (the last such v: rows may be empty)
  while (lo < hi) {
    const int32_t mid = lo + (hi - lo + 1) / 2;
    if (rowptr[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_nbr_deg_sum(int32_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colidx, const int32_t* __restrict__ deg,
                              unsigned long long* __restrict__ s2) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = warp * NDS_CHUNK; c0 < nnz; c0 += nwarps * NDS_CHUNK) {
    const int64_t c1 = c0 + NDS_CHUNK < nnz ? c0 + NDS_CHUNK : nnz;
    int32_t r = row_of_entry(rowptr, 0, n - 1, c0);  // row of the step's first entry (warp-uniform)
    for (int64_t e0 = c0; e0 < c1; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool ok = e < c1;
      unsigned long long val = ok ? (unsigned long long)deg[colidx[e]] : 0ull;
      // end of row r + k in lane k; the count of ends <= e is the lane's row offset
      const int32_t rk = r + 1 + lane;
      const int64_t endk = rk <= n ? rowptr[rk] : INT64_MAX;
      int32_t row = r;
      if (__shfl_sync(NDS_FULL, endk, 0) <= e0 + 31) {  // the step crosses a row end
        int32_t cnt = 0;
#pragma unroll
        for (int b = 16; b >= 1; b >>= 1) {
          const int64_t probe = __shfl_sync(NDS_FULL, endk, cnt + b - 1);
          if (probe <= e) cnt += b;
        }
        if (__shfl_sync(NDS_FULL, endk, cnt) <= e) ++cnt;
        row = cnt < 32 ? r + cnt : row_of_entry(rowptr, r + 32, n - 1, e);
      }
      // segmented inclusive sum over lanes of the same row (rows do not decrease with the lane)
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long ov = __shfl_up_sync(NDS_FULL, val, d);
        const int32_t orow = __shfl_up_sync(NDS_FULL, row, d);
        if (lane >= d && orow == row) val += ov;
      }
      const int32_t nrow = __shfl_down_sync(NDS_FULL, row, 1);
      const bool nok = __shfl_down_sync(NDS_FULL, ok ? 1 : 0, 1) != 0;
      if (ok && val != 0ull && (lane == 31 || !nok || nrow != row)) atomicAdd(&s2[row], val);
      r = __shfl_sync(NDS_FULL, row, 31);
    }
  }
}

__global__ void k_features(int32_t n, double alpha_s, const double* __restrict__ alpha_v,
                           const int32_t* __restrict__ deg, const double* __restrict__ dw,
                           const unsigned long long* __restrict__ s2, float4* __restrict__ X) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    // FP32 logarithms (GB300's FP64 rate made the FP64 ones the cost of the
    // feature pass); the inputs are rounded to FP32 first
    const double alpha = alpha_v ? alpha_v[v] : alpha_s;
    X[v] = make_float4(log1pf((float)deg[v]), log1pf((float)(alpha * dw[v])), log1pf((float)s2[v]),
                       logf((float)alpha));
  }
}

__device__ __forceinline__ void load_params(const float* __restrict__ params, float* sw) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sw[i] = bf16r(params[i]);
  __syncthreads();
}

// z = w2 . relu(W1 x + b1) + b2 with the (BF16-valued) weights in shared memory
__device__ __forceinline__ float mlp_z(const float* sw, const float4& x) {
  float z = sw[OFF_B2];
#pragma unroll 8
  for (int j = 0; j < HID; ++j) {
    const float4 w = *reinterpret_cast<const float4*>(sw + OFF_W1 + j * NF);  // one 16-byte load
    float pre = sw[OFF_B1 + j];
    pre = fmaf(w.x, x.x, pre);
    pre = fmaf(w.y, x.y, pre);
    pre = fmaf(w.z, x.z, pre);
    pre = fmaf(w.w, x.w, pre);
    z = fmaf(sw[OFF_W2 + j], fmaxf(pre, 0.0f), z);
  }
  return z;
}

__global__ void __launch_bounds__(MLP_T) k_mlp_forward(int32_t n, const float4* __restrict__ X,
                                                       const uint4* __restrict__ rinfo,
                                                       const float* __restrict__ params, float* __restrict__ gout) {
  __shared__ __align__(16) float sw[NPARAM];
  load_params(params, sw);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float z = mlp_z(sw, X[v]);
    const float s = 1.0f / (1.0f + expf(-z));
    const float p = (float)p_of(rinfo[v]);
    gout[v] = p + (1.0f - p) * s;
  }
}

// Loss and gradient, per-block partials (fixed order, deterministic).
// Pass over tiles of MLP_T vertices: thread t runs the forward pass of vertex
// t of the tile and its dL/dz; then thread j accumulates the gradient of
// hidden unit j over the tile's vertices in order.
__global__ void __launch_bounds__(MLP_T) k_mlp_grad(int32_t n, const float4* __restrict__ X,
                                                    const uint4* __restrict__ rinfo, const float* __restrict__ y,
                                                    const float* __restrict__ params, float inv_n,
                                                    float* __restrict__ gpart, double* __restrict__ lpart) {
  __shared__ __align__(16) float sw[NPARAM];
  __shared__ float4 sx[MLP_T];
  __shared__ float sdz[MLP_T];
  __shared__ double sl[MLP_T];
  load_params(params, sw);
  const int j = threadIdx.x;
  float gW0 = 0.f, gW1 = 0.f, gW2 = 0.f, gW3 = 0.f, gb1 = 0.f, gw2 = 0.f, gb2 = 0.f;
  double lsum = 0.0;
  const float* wj = sw + OFF_W1 + j * NF;
  for (int64_t base = (int64_t)blockIdx.x * MLP_T; base < n; base += (int64_t)gridDim.x * MLP_T) {
    const int64_t v = base + j;
    float dz = 0.0f;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v < n) {
      x = X[v];
      const float z = mlp_z(sw, x);
      const float s = 1.0f / (1.0f + expf(-z));
      const float p = (float)p_of(rinfo[v]);
      const float g = p + (1.0f - p) * s;
      const float r = g - y[v];
      lsum += (double)r * (double)r;
      dz = 2.0f * r * inv_n * (1.0f - p) * s * (1.0f - s);
    }
    sx[j] = x;
    sdz[j] = dz;
    __syncthreads();
    const int cnt = (n - base) < (int64_t)MLP_T ? (int)(n - base) : MLP_T;
    for (int i = 0; i < cnt; ++i) {
      const float4 xi = sx[i];
      const float dzi = sdz[i];
      float pre = sw[OFF_B1 + j];
      pre = fmaf(wj[0], xi.x, pre);
      pre = fmaf(wj[1], xi.y, pre);
      pre = fmaf(wj[2], xi.z, pre);
      pre = fmaf(wj[3], xi.w, pre);
      if (pre > 0.0f) {
        gw2 = fmaf(dzi, pre, gw2);
        const float dpre = dzi * sw[OFF_W2 + j];
        gW0 = fmaf(dpre, xi.x, gW0);
        gW1 = fmaf(dpre, xi.y, gW1);
        gW2 = fmaf(dpre, xi.z, gW2);
        gW3 = fmaf(dpre, xi.w, gW3);
        gb1 += dpre;
      }
      if (j == 0) gb2 += dzi;
    }
    __syncthreads();
  }
  // parameter-major partials: gpart[i * nb + block] (the reduction reads
  // each parameter's partials contiguously)
  const size_t nb = gridDim.x, b = blockIdx.x;
  gpart[(size_t)(OFF_W1 + j * NF + 0) * nb + b] = gW0;
  gpart[(size_t)(OFF_W1 + j * NF + 1) * nb + b] = gW1;
  gpart[(size_t)(OFF_W1 + j * NF + 2) * nb + b] = gW2;
  gpart[(size_t)(OFF_W1 + j * NF + 3) * nb + b] = gW3;
  gpart[(size_t)(OFF_B1 + j) * nb + b] = gb1;
  gpart[(size_t)(OFF_W2 + j) * nb + b] = gw2;
  if (j == 0) gpart[(size_t)OFF_B2 * nb + b] = gb2;
  sl[j] = lsum;
  __syncthreads();
  for (int s = MLP_T / 2; s > 0; s >>= 1) {
    if (j < s) sl[j] += sl[j + s];
    __syncthreads();
  }
  if (j == 0) lpart[blockIdx.x] = sl[0];
}

// One block per parameter (block NPARAM: the loss): the block's threads sum
// strided runs of the partials, then a fixed-order tree in shared memory, so
// the result is deterministic.  out = (accumulate ? out : 0) + weight * sum.
constexpr int RED_T = 256;
__global__ void __launch_bounds__(RED_T) k_mlp_grad_reduce(const float* __restrict__ gpart,
                                                           const double* __restrict__ lpart, int nb, double inv_n,
                                                           float weight, int accumulate, float* __restrict__ grad,
                                                           float* __restrict__ loss) {
  __shared__ double red[RED_T];
  const int i = blockIdx.x;
  double s = 0.0;
  if (i < NPARAM) {
    for (int b = threadIdx.x; b < nb; b += RED_T) s += (double)gpart[(size_t)i * nb + b];
  } else {
    for (int b = threadIdx.x; b < nb; b += RED_T) s += lpart[b];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = RED_T / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (i < NPARAM) {
    const float v = weight * (float)red[0];
    grad[i] = accumulate ? grad[i] + v : v;
  } else if (loss != nullptr) {
    const float v = weight * (float)(red[0] * inv_n);
    *loss = accumulate ? *loss + v : v;
  }
}

__global__ void k_adam(int32_t count, float* __restrict__ params, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static int mlp_blocks(int32_t n) {
  int64_t b = ((int64_t)n + MLP_T - 1) / MLP_T;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

}  // namespace fcx

using namespace fcx;

extern "C" int32_t fc_mlp_param_count(void) { return NPARAM; }

extern "C" fc_status fc_vertex_features(fc_graph* g, int32_t alpha_idx, float* X, void* stream) {
  if (g == nullptr || X == nullptr || alpha_idx < 0 || alpha_idx >= g->n_alpha) {
    set_error("fc_vertex_features: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* s2 = nullptr;
  FC_CK(cudaMallocAsync((void**)&s2, (size_t)g->n * sizeof(unsigned long long), st));
  FC_CK(cudaMemsetAsync(s2, 0, (size_t)g->n * sizeof(unsigned long long), st));
  const int64_t chunks = (g->nnz + NDS_CHUNK - 1) / NDS_CHUNK;  // one warp each, 8 warps per block
  if (chunks > 0) {
    const unsigned nb = (unsigned)std::min<int64_t>((chunks + 7) / 8, 152 * 8);
    k_nbr_deg_sum<<<nb, 256, 0, st>>>(g->n, g->nnz, g->rowptr, g->colidx, g->deg, s2);
    FC_LAUNCHED();
  }
  const unsigned fb = (unsigned)std::min<int64_t>(((int64_t)g->n + 255) / 256, 152 * 16);
  k_features<<<fb, 256, 0, st>>>(g->n, g->alphas[alpha_idx], g->alpha_v, g->deg, g->dw, s2, (float4*)X);
  FC_LAUNCHED();
  FC_CK(cudaFreeAsync(s2, st));
  return FC_OK;
}

extern "C" fc_status fc_mlp_forward(fc_graph* g, int32_t alpha_idx, const float* X, const float* params,
                                    float* g_out, void* stream) {
  if (g == nullptr || X == nullptr || params == nullptr || g_out == nullptr || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha) {
    set_error("fc_mlp_forward: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  k_mlp_forward<<<mlp_blocks(g->n), MLP_T, 0, st>>>(g->n, (const float4*)X, g->rowinfo + (size_t)alpha_idx * g->n,
                                                    params, g_out);
  FC_LAUNCHED();
  return FC_OK;
}

extern "C" fc_status fc_mlp_loss_grad_acc(fc_graph* g, int32_t alpha_idx, const float* X, const float* y,
                                          const float* params, float weight, int32_t accumulate, float* grad,
                                          float* loss, void* stream) {
  if (g == nullptr || X == nullptr || y == nullptr || params == nullptr || grad == nullptr || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha || !std::isfinite(weight)) {
    set_error("fc_mlp_loss_grad: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = mlp_blocks(g->n);
  float* gpart = nullptr;
  double* lpart = nullptr;
  FC_CK(cudaMallocAsync((void**)&gpart, (size_t)nb * NPARAM * sizeof(float), st));
  FC_CK(cudaMallocAsync((void**)&lpart, (size_t)nb * sizeof(double), st));
  k_mlp_grad<<<nb, MLP_T, 0, st>>>(g->n, (const float4*)X, g->rowinfo + (size_t)alpha_idx * g->n, y, params,
                                   1.0f / (float)g->n, gpart, lpart);
  FC_LAUNCHED();
  k_mlp_grad_reduce<<<NPARAM + 1, RED_T, 0, st>>>(gpart, lpart, nb, 1.0 / (double)g->n, weight, accumulate ? 1 : 0,
                                                  grad, loss);
  FC_LAUNCHED();
  FC_CK(cudaFreeAsync(gpart, st));
  FC_CK(cudaFreeAsync(lpart, st));
  return FC_OK;
}

extern "C" fc_status fc_mlp_loss_grad(fc_graph* g, int32_t alpha_idx, const float* X, const float* y,
                                      const float* params, float* grad, float* loss, void* stream) {
  return fc_mlp_loss_grad_acc(g, alpha_idx, X, y, params, 1.0f, 0, grad, loss, stream);
}

extern "C" fc_status fc_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t count, int32_t step,
                                 float lr, float beta1, float beta2, float eps, void* stream) {
  if (params == nullptr || grad == nullptr || m == nullptr || v == nullptr || count < 1 || step < 1) {
    set_error("fc_mlp_adam: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float c1 = 1.0f - powf(beta1, (float)step);
  const float c2 = 1.0f - powf(beta2, (float)step);
  k_adam<<<(count + 255) / 256, 256, 0, st>>>(count, params, grad, m, v, lr, beta1, beta2, eps, c1, c2);
  FC_LAUNCHED();
  return FC_OK;
}
