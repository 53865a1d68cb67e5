// Tree-path aggregation over sampled trees: forest roots and depths by BFS
// levels from u*, and root-frequency counts.
//
// In a spanning tree of G* rooted at u*, removing u* leaves a rooted spanning
// forest of G whose roots are the children of u*.  By the matrix-forest
// theorem (Sec. 2), Omega[u, v] is the probability that v's tree of that
// forest is rooted at u, so root frequencies over sampled trees estimate whole
// columns of Omega (the diagonal is Prop. 1's u*-edge frequency), and with them
// pairwise forest distances rho(u, v) = Omega_uu + Omega_vv - 2 Omega_uv
// (Def. 1).
//
// fc_tree_roots: one CTA per tree.  Children lists are built by counting
// (atomic child counts, a block-wide exclusive scan made of warp scans, a
// scatter); the BFS then expands one level at a time, each level's output
// positions again from a block-wide scan of the frontier's child counts.
#include "fc_internal.cuh"

namespace fcx {

constexpr int AG_T = 1024;

// Block-wide exclusive scan of one value per thread (warp shuffles, then a
// scan of the warp totals).  Returns the exclusive prefix; *total gets the sum.
__device__ __forceinline__ int32_t block_exscan(int32_t x, int32_t* total, int32_t* wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t s = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += y;
  }
  if (lane == 31) wsum[wid] = s;
  __syncthreads();
  if (wid == 0) {
    int32_t t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  const int32_t excl = s - x + (wid > 0 ? wsum[wid - 1] : 0);
  *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return excl;
}

// scratch per CTA slot: cnt/off [n+1], fill [n], child [n], front [2][n]
__global__ void __launch_bounds__(AG_T) k_tree_roots(const int32_t* __restrict__ parents, int32_t n, int64_t T,
                                                     int32_t* __restrict__ roots, int32_t* __restrict__ depth,
                                                     int32_t* __restrict__ scratch, uint32_t* err) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t sh_carry, sh_len;
  const size_t sn = (size_t)n;
  int32_t* off = scratch + (size_t)blockIdx.x * (5 * sn + 1);
  int32_t* fill = off + sn + 1;
  int32_t* child = fill + sn;
  int32_t* front0 = child + sn;
  int32_t* front1 = front0 + sn;
  for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
    const int32_t* par = parents + (size_t)t * sn;
    int32_t* rt = roots + (size_t)t * sn;
    int32_t* dp = depth ? depth + (size_t)t * sn : nullptr;
    // child counts
    for (int32_t v = threadIdx.x; v <= n; v += AG_T) off[v] = 0;
    for (int32_t v = threadIdx.x; v < n; v += AG_T) fill[v] = 0;
    __syncthreads();
    for (int32_t v = threadIdx.x; v < n; v += AG_T) {
      const int32_t p = par[v];
      if (p < 0 || p > n || p == v) atomicOr(err, ERR_INVAL);
      else if (p < n) atomicAdd(&off[p], 1);
    }
    __syncthreads();
    // exclusive scan of the counts, chunk by chunk with a running carry
    if (threadIdx.x == 0) sh_carry = 0;
    __syncthreads();
    for (int32_t b0 = 0; b0 <= n; b0 += AG_T) {
      const int32_t v = b0 + threadIdx.x;
      const int32_t x = v <= n ? off[v] : 0;
      int32_t tot = 0;
      const int32_t ex = block_exscan(x, &tot, wsum);
      if (v <= n) off[v] = sh_carry + ex;
      __syncthreads();
      if (threadIdx.x == 0) sh_carry += tot;
      __syncthreads();
    }
    // scatter children
    for (int32_t v = threadIdx.x; v < n; v += AG_T) {
      const int32_t p = par[v];
      if (p >= 0 && p < n && p != v) child[off[p] + atomicAdd(&fill[p], 1)] = v;
    }
    // level 0: the children of u* are their own roots
    if (threadIdx.x == 0) sh_len = 0;
    __syncthreads();
    for (int32_t b0 = 0; b0 < n; b0 += AG_T) {
      const int32_t v = b0 + threadIdx.x;
      const int32_t is_root = (v < n && par[v] == n) ? 1 : 0;
      int32_t tot = 0;
      const int32_t ex = block_exscan(is_root, &tot, wsum);
      if (is_root) {
        front0[sh_len + ex] = v;
        rt[v] = v;
        if (dp) dp[v] = 0;
      }
      __syncthreads();
      if (threadIdx.x == 0) sh_len += tot;
      __syncthreads();
    }
    int32_t len = sh_len;
    int32_t* cur = front0;
    int32_t* nxt = front1;
    int32_t level = 0, seen = len;
    while (len > 0) {
      ++level;
      if (threadIdx.x == 0) sh_len = 0;
      __syncthreads();
      for (int32_t b0 = 0; b0 < len; b0 += AG_T) {
        const int32_t i = b0 + threadIdx.x;
        int32_t f = -1, cnt = 0, c0 = 0;
        if (i < len) {
          f = cur[i];
          c0 = off[f];
          cnt = off[f + 1] - c0;
        }
        int32_t tot = 0;
        const int32_t ex = block_exscan(cnt, &tot, wsum);
        const int32_t base = sh_len;
        for (int32_t j = 0; j < cnt; ++j) {
          const int32_t c = child[c0 + j];
          nxt[base + ex + j] = c;
          rt[c] = rt[f];
          if (dp) dp[c] = level;
        }
        __syncthreads();
        if (threadIdx.x == 0) sh_len += tot;
        __syncthreads();
      }
      len = sh_len;
      seen += len;
      int32_t* tmp = cur;
      cur = nxt;
      nxt = tmp;
      if (level > n) break;
    }
    if (threadIdx.x == 0 && seen != n) atomicOr(err, ERR_INVAL);  // not a tree rooted at u*
    __syncthreads();
  }
}

// counts[q][v] += #{t : roots[t][v] == queries[q]}; qidx[u] = q or -1
__global__ void k_root_counts(const int32_t* __restrict__ roots, int32_t n, int64_t T,
                              const int32_t* __restrict__ qidx, uint32_t* __restrict__ counts) {
  const size_t total = (size_t)T * (size_t)n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int32_t r = roots[i];
    if (r < 0 || r >= n) continue;
    const int32_t q = qidx[r];
    if (q >= 0) atomicAdd(&counts[(size_t)q * n + (i % (size_t)n)], 1u);
  }
}

__global__ void k_qidx(int32_t n, const int32_t* __restrict__ queries, int32_t k, int32_t* __restrict__ qidx,
                       uint32_t* err) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) {
    const int32_t u = queries[i];
    if (u < 0 || u >= n) atomicOr(err, ERR_INVAL);
    else atomicCAS(&qidx[u], -1, i);  // first query wins for duplicates
  }
}

}  // namespace fcx

using namespace fcx;

extern "C" fc_status fc_tree_roots(const int32_t* parents, int32_t n, int64_t T, int32_t* roots, int32_t* depth,
                                   void* stream) {
  if (parents == nullptr || roots == nullptr || n < 1 || T < 0) {
    set_error("fc_tree_roots: bad argument");
    return FC_EINVAL;
  }
  if (T == 0) return FC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int nsm = 0, dev = 0;
  FC_CK(cudaGetDevice(&dev));
  FC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t grid = std::min<int64_t>(T, (int64_t)nsm * 2);
  int32_t* scratch = nullptr;
  uint32_t* err = nullptr;
  FC_CK(cudaMallocAsync((void**)&scratch, (size_t)grid * (5 * (size_t)n + 1) * sizeof(int32_t), st));
  FC_CK(cudaMallocAsync((void**)&err, sizeof(uint32_t), st));
  FC_CK(cudaMemsetAsync(err, 0, sizeof(uint32_t), st));
  k_tree_roots<<<(unsigned)grid, AG_T, 0, st>>>(parents, n, T, roots, depth, scratch, err);
  FC_LAUNCHED();
  uint32_t herr = 0;
  FC_CK(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  FC_CK(cudaFreeAsync(scratch, st));
  FC_CK(cudaFreeAsync(err, st));
  FC_CK(cudaStreamSynchronize(st));
  if (herr) {
    set_error("fc_tree_roots: parents do not form spanning trees rooted at u* = n");
    return FC_EINVAL;
  }
  return FC_OK;
}

extern "C" fc_status fc_root_counts(const int32_t* roots, int32_t n, int64_t T, const int32_t* queries, int32_t k,
                                    uint32_t* counts, void* stream) {
  if (roots == nullptr || queries == nullptr || counts == nullptr || n < 1 || T < 0 || k < 1) {
    set_error("fc_root_counts: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* qidx = nullptr;
  uint32_t* err = nullptr;
  FC_CK(cudaMallocAsync((void**)&qidx, (size_t)n * sizeof(int32_t), st));
  FC_CK(cudaMallocAsync((void**)&err, sizeof(uint32_t), st));
  FC_CK(cudaMemsetAsync(qidx, 0xff, (size_t)n * sizeof(int32_t), st));
  FC_CK(cudaMemsetAsync(err, 0, sizeof(uint32_t), st));
  k_qidx<<<(k + 255) / 256, 256, 0, st>>>(n, queries, k, qidx, err);
  FC_LAUNCHED();
  if (T > 0) {
    const size_t total = (size_t)T * (size_t)n;
    const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 64);
    k_root_counts<<<blocks, 256, 0, st>>>(roots, n, T, qidx, counts);
    FC_LAUNCHED();
  }
  uint32_t herr = 0;
  FC_CK(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  FC_CK(cudaFreeAsync(qidx, st));
  FC_CK(cudaFreeAsync(err, st));
  FC_CK(cudaStreamSynchronize(st));
  if (herr) {
    set_error("fc_root_counts: query vertex out of range");
    return FC_EINVAL;
  }
  return FC_OK;
}
