// Tree-path aggregation over sampled trees: forest roots and depths, and
// root-frequency counts.
//
// In a spanning tree of G* rooted at u*, removing u* leaves a rooted spanning
// forest of G whose roots are the children of u*.  By the matrix-forest
// theorem (Sec. 2), Omega[u, v] is the probability that v's tree of that
// forest is rooted at u, so root frequencies over sampled trees estimate whole
// columns of Omega (the diagonal is Prop. 1's u*-edge frequency), and with them
// pairwise forest distances rho(u, v) = Omega_uu + Omega_vv - 2 Omega_uv
// (Def. 1).
//
// fc_tree_roots: pointer jumping over all trees at once.  Every node holds a
// 64-bit word {ancestor, distance to it}: a root (parent u*) points at itself
// at distance 0, any other node at its parent at distance 1.  A round
// replaces each word {a, d} by {ancestor of a, d + a's distance}; a node
// pointing at a root no longer changes, so O(log depth) rounds end with every
// node at its root and depth.  Words are read and written whole, so a node
// may read a word of this round or the last one.  A parent cycle never
// reaches a root and is caught by the round limit and the final check.
// (A first version took one CTA per tree with children lists and BFS levels;
// its per-tree scratch, touched at random, moved 60x the algorithmic bytes.)
#include "fc_internal.cuh"

namespace fcx {

constexpr int AG_T = 256;

__device__ __forceinline__ unsigned long long rw_pack(int32_t a, int32_t d) {
  return (unsigned long long)(uint32_t)a | ((unsigned long long)(uint32_t)d << 32);
}

__global__ void k_roots_init(const int32_t* __restrict__ parents, int32_t n, int64_t N,
                             unsigned long long* __restrict__ jw, uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = (int32_t)(i % n);
    const int32_t p = parents[i];
    if (p < 0 || p > n || p == v) {
      atomicOr(err, ERR_INVAL);
      jw[i] = rw_pack(v, 0);
    } else {
      jw[i] = p == n ? rw_pack(v, 0) : rw_pack(p, 1);
    }
  }
}

__global__ void __launch_bounds__(AG_T) k_roots_jump(int32_t n, int64_t N, unsigned long long* jw,
                                                     uint32_t* changed) {
  volatile unsigned long long* jv = jw;
  bool any = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long w = jv[i];
    const int32_t a = (int32_t)(uint32_t)w;
    const int64_t base = i - i % n;
    const unsigned long long wa = jv[base + a];
    const int32_t aa = (int32_t)(uint32_t)wa;
    if (aa != a) {
      jv[i] = rw_pack(aa, (int32_t)((uint32_t)(w >> 32) + (uint32_t)(wa >> 32)));
      any = true;
    }
  }
  if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(changed, 1u);
}

__global__ void k_roots_out(const int32_t* __restrict__ parents, int32_t n, int64_t N,
                            const unsigned long long* __restrict__ jw, int32_t* __restrict__ roots,
                            int32_t* __restrict__ depth, uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long w = jw[i];
    const int32_t r = (int32_t)(uint32_t)w;
    const int64_t base = i - i % n;
    if (r < 0 || r >= n || parents[base + r] != n) atomicOr(err, ERR_INVAL);  // not a tree rooted at u*
    roots[i] = r;
    if (depth) depth[i] = (int32_t)(w >> 32);
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
  const int64_t N = T * (int64_t)n;
  const unsigned blocks = (unsigned)std::min<int64_t>((N + AG_T - 1) / AG_T, (int64_t)nsm * 16);
  unsigned long long* jw = nullptr;
  uint32_t* flags = nullptr;  // [0] error, [1] changed in this round
  FC_CK(cudaMallocAsync((void**)&jw, (size_t)N * sizeof(unsigned long long), st));
  FC_CK(cudaMallocAsync((void**)&flags, 2 * sizeof(uint32_t), st));
  FC_CK(cudaMemsetAsync(flags, 0, 2 * sizeof(uint32_t), st));
  k_roots_init<<<blocks, AG_T, 0, st>>>(parents, n, N, jw, flags);
  FC_LAUNCHED();
  uint32_t h[2] = {0u, 1u};
  int round = 0;
  // depth < n < 2^31 needs at most 32 rounds; more means a parent cycle
  for (; round < 40 && h[0] == 0u && h[1] != 0u; ++round) {
    FC_CK(cudaMemsetAsync(flags + 1, 0, sizeof(uint32_t), st));
    k_roots_jump<<<blocks, AG_T, 0, st>>>(n, N, jw, flags + 1);
    FC_LAUNCHED();
    FC_CK(cudaMemcpyAsync(h, flags, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    FC_CK(cudaStreamSynchronize(st));
  }
  if (h[0] == 0u) {
    k_roots_out<<<blocks, AG_T, 0, st>>>(parents, n, N, jw, roots, depth, flags);
    FC_LAUNCHED();
    FC_CK(cudaMemcpyAsync(h, flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  }
  FC_CK(cudaFreeAsync(jw, st));
  FC_CK(cudaFreeAsync(flags, st));
  FC_CK(cudaStreamSynchronize(st));
  if (h[0] != 0u || h[1] != 0u) {
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
