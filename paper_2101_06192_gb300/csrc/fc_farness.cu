// Combination (Algorithm 1's fill step, control variate), forest farness
// (Eq. 3), forest closeness (Def. 2), exact u*-selection probabilities, and
// the top-k ranking (Sec. 6.1).
#include <algorithm>
#include <vector>

#include "fc_internal.cuh"

namespace fcx {

// Record msg as the last error and return FC_EINVAL.
static inline fc_status invalid(const char* msg) {
  set_error(msg);
  return FC_EINVAL;
}

constexpr int RED_THREADS = 256;

// p_v = T_v / 2^53 (exact: T_v <= 2^53)
__device__ __forceinline__ double p_from_rowinfo(const uint4& ri) {
  const uint64_t T = (uint64_t)ri.z | ((uint64_t)ri.w << 32);
  return (double)T * 0x1.0p-53;
}

// Pass 1: d_v and per-block partial sums of d (fixed-order tree reduction).
__global__ void k_combine(int32_t n, const uint32_t* __restrict__ R, const uint32_t* __restrict__ C,
                          const float* __restrict__ gpred, const uint4* __restrict__ rinfo,
                          const double* __restrict__ xpiv, double inv_tau, double* __restrict__ diag,
                          double* __restrict__ partial) {
  __shared__ double red[RED_THREADS];
  const int64_t v = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x;
  double d = 0.0;
  if (v < n) {
    d = (double)R[v] * inv_tau;
    if (xpiv != nullptr) {
      // fill step: R/tau - x(u*) + 2 x(v) = diag(L*^+) on V; add back (n+2)/(n+1)^2
      const double n1 = (double)n + 1.0;
      d = d - xpiv[n] + 2.0 * xpiv[v] + ((double)n + 2.0) / (n1 * n1);
    }
    if (C != nullptr) {
      const double p = p_from_rowinfo(rinfo[v]);
      if (p < 1.0) {
        // clip(g, p, 1); a prediction that is not a number counts as p (so
        // every g_pred, NaN included, leaves the estimator unbiased)
        double gg = (double)gpred[v];
        gg = (gg >= p) ? fmin(gg, 1.0) : p;
        const double beta = (1.0 - gg) / (1.0 - p);
        d = d - beta * ((double)C[v] * inv_tau - p);
      }
    }
    diag[v] = d;
  }
  red[threadIdx.x] = d;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Pass 2: single block sums the partials in a fixed order.
__global__ void k_sum_partials(const double* __restrict__ partial, int64_t m, double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += 1024) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 512; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_farness(int32_t n, const double* __restrict__ diag, const double* __restrict__ trace,
                          double* __restrict__ farness, double* __restrict__ closeness) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double f = (double)n * diag[v] + *trace - 2.0;  // Eq. 3
  if (farness) farness[v] = f;
  if (closeness) closeness[v] = (double)n / f;         // Def. 2
}

// Batch of graphs: per-graph trace (one block per graph, fixed order) and
// farness with that graph's n and trace.
__global__ void k_seg_trace(const int64_t* __restrict__ voff, const double* __restrict__ diag,
                            double* __restrict__ tr) {
  __shared__ double red[RED_THREADS];
  const int gi = blockIdx.x;
  double s = 0.0;
  for (int64_t v = voff[gi] + threadIdx.x; v < voff[gi + 1]; v += RED_THREADS) s += diag[v];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = RED_THREADS / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) tr[gi] = red[0];
}

__global__ void k_farness_seg(int32_t n, const int32_t* __restrict__ gid, const int64_t* __restrict__ voff,
                              const double* __restrict__ diag, const double* __restrict__ tr,
                              double* __restrict__ farness, double* __restrict__ closeness) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t gi = gid[v];
  const double ng = (double)(voff[gi + 1] - voff[gi]);
  const double f = ng * diag[v] + tr[gi] - 2.0;  // Eq. 3 within the graph
  if (farness) farness[v] = f;
  if (closeness) closeness[v] = ng / f;          // Def. 2
}

// diag_v = visits[v] / (tau deg*(v)), deg*(v) = fl(1 + fl(alpha d_w(v)))
__global__ void k_visit_diag(int32_t n, const unsigned long long* __restrict__ visits, double alpha_s,
                             const double* __restrict__ alpha_v, const double* __restrict__ dw, double tau,
                             double* __restrict__ diag) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double a = alpha_v ? alpha_v[v] : alpha_s;
  diag[v] = __ddiv_rn((double)visits[v], __dmul_rn(tau, deg_star(a, dw[v])));
}

__global__ void k_p_root(int32_t n, const uint4* __restrict__ rinfo, double* __restrict__ p) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) p[v] = p_from_rowinfo(rinfo[v]);
}

// ---------------------------------------------------------------------------
// top-k: stable LSD radix sort of (order-preserving 64-bit key of diag, id).
// Inputs are in id order, so equal keys keep ascending ids.
// ---------------------------------------------------------------------------
constexpr int TK_TILE = 1024;

// Order-preserving key: -0.0 and +0.0 compare equal (ties then go by id) and
// every NaN sorts after +inf.
__device__ __forceinline__ uint64_t ordered_key(double d) {
  if (d == 0.0) d = 0.0;
  if (isnan(d)) return ~0ull;
  uint64_t u = (uint64_t)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_tk_init(int32_t n, const double* __restrict__ diag, uint64_t* __restrict__ keys,
                          int32_t* __restrict__ vals) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) {
    keys[v] = ordered_key(diag[v]);
    vals[v] = (int32_t)v;
  }
}

__global__ void k_tk_hist(int32_t n, const uint64_t* __restrict__ keys, int shift, uint32_t* __restrict__ hist,
                          int32_t nblk) {
  __shared__ uint32_t cnt[256];
  const int lane = threadIdx.x;
  for (int d = lane; d < 256; d += 32) cnt[d] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * TK_TILE;
  for (int c = 0; c < TK_TILE / 32; ++c) {
    const int64_t i = base + c * 32 + lane;
    if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 255u], 1u);
  }
  __syncwarp();
  for (int d = lane; d < 256; d += 32) hist[(int64_t)d * nblk + blockIdx.x] = cnt[d];
}

__global__ void k_tk_scatter(int32_t n, const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int shift,
                             const uint32_t* __restrict__ offs, int32_t nblk) {
  __shared__ uint32_t run[256];
  const int lane = threadIdx.x;
  for (int d = lane; d < 256; d += 32) run[d] = offs[(int64_t)d * nblk + blockIdx.x];
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * TK_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < TK_TILE / 32; ++c) {
    const int64_t i = base + c * 32 + lane;
    const bool valid = i < n;
    uint64_t key = 0;
    int32_t val = 0;
    uint32_t d = 256u + lane;
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = (uint32_t)(key >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt);
    if (valid) {
      const uint32_t pos = run[d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) run[d] += __popc(peers);
    __syncwarp();
  }
}

// per-block sums of diag in the same fixed tree order as k_combine's
__global__ void k_block_sums(int32_t n, const double* __restrict__ diag, double* __restrict__ partial) {
  __shared__ double red[RED_THREADS];
  const int64_t v = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x;
  red[threadIdx.x] = v < n ? diag[v] : 0.0;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace fcx

using namespace fcx;

extern "C" fc_status fc_forest_farness(fc_graph* g, int32_t alpha_idx, const uint32_t* R, const uint32_t* C,
                                       const float* g_pred, const double* x_pivot, int64_t tau,
                                       double* diag_out, double* farness_out, double* closeness_out,
                                       void* stream) {
  if (g == nullptr || R == nullptr || diag_out == nullptr || tau < 1 || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha || ((C == nullptr) != (g_pred == nullptr))) {
    set_error("fc_forest_farness: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  const int64_t nb = (n + RED_THREADS - 1) / RED_THREADS;
  double* partial = nullptr;
  FC_CK(cudaMallocAsync((void**)&partial, (nb + 1) * sizeof(double), st));
  const uint4* rinfo = g->rowinfo + (size_t)alpha_idx * n;
  k_combine<<<(unsigned)nb, RED_THREADS, 0, st>>>(n, R, C, g_pred, rinfo, x_pivot, 1.0 / (double)tau, diag_out,
                                                  partial);
  FC_LAUNCHED();
  if (g->num_graphs > 0) {
    double* tr = nullptr;
    FC_CK(cudaMallocAsync((void**)&tr, (size_t)g->num_graphs * sizeof(double), st));
    k_seg_trace<<<g->num_graphs, RED_THREADS, 0, st>>>(g->voff, diag_out, tr);
    FC_LAUNCHED();
    if (farness_out || closeness_out) {
      k_farness_seg<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, g->gid, g->voff, diag_out, tr, farness_out,
                                                                 closeness_out);
      FC_LAUNCHED();
    }
    FC_CK(cudaFreeAsync(tr, st));
    FC_CK(cudaFreeAsync(partial, st));
    return FC_OK;
  }
  k_sum_partials<<<1, 1024, 0, st>>>(partial, nb, partial + nb);
  FC_LAUNCHED();
  if (farness_out || closeness_out) {
    k_farness<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, diag_out, partial + nb, farness_out, closeness_out);
    FC_LAUNCHED();
  }
  FC_CK(cudaFreeAsync(partial, st));
  return FC_OK;
}

extern "C" fc_status fc_farness_from_diag(fc_graph* g, const double* diag, double* farness_out,
                                          double* closeness_out, void* stream) {
  if (g == nullptr || diag == nullptr) {
    set_error("fc_farness_from_diag: bad argument");
    return FC_EINVAL;
  }
  if (farness_out == nullptr && closeness_out == nullptr) return FC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  if (g->num_graphs > 0) {
    double* tr = nullptr;
    FC_CK(cudaMallocAsync((void**)&tr, (size_t)g->num_graphs * sizeof(double), st));
    k_seg_trace<<<g->num_graphs, RED_THREADS, 0, st>>>(g->voff, diag, tr);
    FC_LAUNCHED();
    k_farness_seg<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, g->gid, g->voff, diag, tr, farness_out,
                                                               closeness_out);
    FC_LAUNCHED();
    FC_CK(cudaFreeAsync(tr, st));
    return FC_OK;
  }
  const int64_t nb = (n + RED_THREADS - 1) / RED_THREADS;
  double* partial = nullptr;
  FC_CK(cudaMallocAsync((void**)&partial, (nb + 1) * sizeof(double), st));
  k_block_sums<<<(unsigned)nb, RED_THREADS, 0, st>>>(n, diag, partial);
  FC_LAUNCHED();
  k_sum_partials<<<1, 1024, 0, st>>>(partial, nb, partial + nb);
  FC_LAUNCHED();
  k_farness<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, diag, partial + nb, farness_out, closeness_out);
  FC_LAUNCHED();
  FC_CK(cudaFreeAsync(partial, st));
  return FC_OK;
}

extern "C" fc_status fc_p_root(fc_graph* g, int32_t alpha_idx, double* p_out, void* stream) {
  if (g == nullptr || p_out == nullptr || alpha_idx < 0 || alpha_idx >= g->n_alpha)
    return fcx::invalid("fc_p_root: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  k_p_root<<<(unsigned)((g->n + 255) / 256), 256, 0, st>>>(g->n, g->rowinfo + (size_t)alpha_idx * g->n, p_out);
  FC_LAUNCHED();
  return FC_OK;
}

extern "C" fc_status fc_top_k(const double* diag, int32_t n, int32_t k, int32_t* idx_out, void* stream) {
  if (diag == nullptr || idx_out == nullptr || n < 1 || k < 1 || k > n) {
    set_error("fc_top_k: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t nblk = (n + TK_TILE - 1) / TK_TILE;
  const int64_t hlen = (int64_t)256 * nblk;
  uint64_t *k0 = nullptr, *k1 = nullptr;
  int32_t *v0 = nullptr, *v1 = nullptr;
  uint32_t *hist = nullptr, *offs = nullptr;
  FC_CK(cudaMallocAsync((void**)&k0, (size_t)n * 8, st));
  FC_CK(cudaMallocAsync((void**)&k1, (size_t)n * 8, st));
  FC_CK(cudaMallocAsync((void**)&v0, (size_t)n * 4, st));
  FC_CK(cudaMallocAsync((void**)&v1, (size_t)n * 4, st));
  FC_CK(cudaMallocAsync((void**)&hist, (size_t)hlen * 4, st));
  FC_CK(cudaMallocAsync((void**)&offs, (size_t)hlen * 4, st));
  k_tk_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, diag, k0, v0);
  FC_LAUNCHED();
  uint64_t* kin = k0;
  uint64_t* kout = k1;
  int32_t* vin = v0;
  int32_t* vout = v1;
  for (int pass = 0; pass < 8; ++pass) {
    k_tk_hist<<<nblk, 32, 0, st>>>(n, kin, 8 * pass, hist, nblk);
    FC_LAUNCHED();
    const fc_status r = exclusive_scan(hist, offs, hlen, st);
    if (r != FC_OK) return r;
    k_tk_scatter<<<nblk, 32, 0, st>>>(n, kin, vin, kout, vout, 8 * pass, offs, nblk);
    FC_LAUNCHED();
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  FC_CK(cudaMemcpyAsync(idx_out, vin, (size_t)k * 4, cudaMemcpyDeviceToDevice, st));
  FC_CK(cudaFreeAsync(k0, st));
  FC_CK(cudaFreeAsync(k1, st));
  FC_CK(cudaFreeAsync(v0, st));
  FC_CK(cudaFreeAsync(v1, st));
  FC_CK(cudaFreeAsync(hist, st));
  FC_CK(cudaFreeAsync(offs, st));
  FC_CK(cudaStreamSynchronize(st));
  return FC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of fc_forest_farness.  The per-block partial sums
// and the trace live in a file-scope device array instead of stream-ordered
// pool memory.  Host code must not pass the array's name to a kernel (on the
// host it is only a stand-in symbol), so its device address on the current
// device is looked up with cudaGetSymbolAddress at every call (a host-side
// lookup; nothing cached, so a reset device or a reloaded module is no issue).
// ---------------------------------------------------------------------------
namespace fcx {
constexpr int32_t NOALLOC_MAX_N = 1 << 22;
constexpr int64_t NOALLOC_MAX_BLOCKS = (NOALLOC_MAX_N + RED_THREADS - 1) / RED_THREADS;
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS + 1];

static fc_status noalloc_scratch(double** out) {
  void* p = nullptr;
  FC_CK(cudaGetSymbolAddress(&p, g_noalloc_partials));
  *out = (double*)p;
  return FC_OK;
}
}  // namespace fcx

extern "C" fc_status fc_forest_farness_noalloc(fc_graph* g, int32_t alpha_idx, const uint32_t* R,
                                               const uint32_t* C, const float* g_pred, const double* x_pivot,
                                               int64_t tau, double* diag_out, double* farness_out,
                                               double* closeness_out, void* stream) {
  if (g == nullptr || R == nullptr || diag_out == nullptr || tau < 1 || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha || ((C == nullptr) != (g_pred == nullptr))) {
    set_error("fc_forest_farness_noalloc: bad argument");
    return FC_EINVAL;
  }
  if (g->num_graphs > 0) {
    set_error("fc_forest_farness_noalloc: batches of graphs need per-graph traces; use fc_forest_farness");
    return FC_EINVAL;
  }
  if (g->n > NOALLOC_MAX_N) {
    set_error("fc_forest_farness_noalloc: n exceeds the fixed scratch capacity of 4194304 vertices; "
              "use fc_forest_farness");
    return FC_EINVAL;
  }
  int dev = -1;
  FC_CK(cudaGetDevice(&dev));
  if (dev != g->device) {
    set_error("fc_forest_farness_noalloc: the graph's device is not the current device");
    return FC_EINVAL;
  }
  double* partial = nullptr;
  const fc_status s = noalloc_scratch(&partial);
  if (s != FC_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  const int64_t nb = (n + RED_THREADS - 1) / RED_THREADS;
  const uint4* rinfo = g->rowinfo + (size_t)alpha_idx * n;
  // k_combine writes partial[0, nb) and k_sum_partials writes partial[nb]
  // before anything reads them, so no clearing is needed between calls.
  k_combine<<<(unsigned)nb, RED_THREADS, 0, st>>>(n, R, C, g_pred, rinfo, x_pivot, 1.0 / (double)tau, diag_out,
                                                  partial);
  FC_LAUNCHED();
  k_sum_partials<<<1, 1024, 0, st>>>(partial, nb, partial + nb);
  FC_LAUNCHED();
  if (farness_out || closeness_out) {
    k_farness<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, diag_out, partial + nb, farness_out, closeness_out);
    FC_LAUNCHED();
  }
  return FC_OK;
}

extern "C" fc_status fc_visit_diag(fc_graph* g, int32_t alpha_idx, const uint64_t* visits, int64_t tau,
                                   double* diag_out, void* stream) {
  if (g == nullptr || visits == nullptr || diag_out == nullptr || tau < 1 || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha || g->root >= 0) {
    set_error("fc_visit_diag: bad argument (a graph from fc_build_augmented or fc_build_batch)");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  k_visit_diag<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      n, (const unsigned long long*)visits + (size_t)alpha_idx * n, g->alphas[alpha_idx],
      g->num_graphs > 0 ? g->alpha_v : nullptr, g->dw, (double)tau, diag_out);
  FC_LAUNCHED();
  return FC_OK;
}
