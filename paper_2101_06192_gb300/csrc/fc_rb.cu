// Rao-Blackwellised estimate of diag(Omega) from sampled trees: an estimator
// on the same samples as Prop. 1 (not in the paper).
//
// With the parents of all vertices but v fixed, the vertices whose path to
// u* runs through v (v's subtree S(v), v included) are fixed, and v's parent
// can be u* (edge weight 1) or any neighbour w outside S(v) (edge weight
// alpha w_vw); every choice gives a spanning tree of G* whose weight is the
// same product times that edge's weight.  So
//     P(parent(v) = u* | the other parents) = 1 / (1 + alpha sum_{w in N(v)\S(v)} w_vw),
// and its average over trees is unbiased for Omega[v, v] with at most the
// variance of the indicator.  w in S(v) iff tin[v] <= tin[w] < tin[v] +
// size[v] for a preorder numbering tin and subtree sizes.  The sum runs over
// v's CSR row in order in FP64 and the value 1 / (1 + alpha s) is rounded
// once per operation; per tree it is added in fixed point, floor(value *
// 2^48 + 1/2), so totals do not depend on the order of the additions.
//
// One cooperative kernel handles a chunk of trees with every resident CTA;
// grid-wide barriers separate the phases: child counts (with validation), a
// grid-wide exclusive scan, children and roots, level-synchronous BFS from
// the roots, subtree sizes bottom-up, preorder numbers top-down, and one
// thread per (tree, vertex) scanning the vertex's row.  Every loop bound and
// every early exit is read from global memory after a barrier, so all CTAs
// take the same path through the barriers.
#include <cooperative_groups.h>

#include <algorithm>

#include "fc_internal.cuh"

namespace cg = cooperative_groups;

namespace fcx {

namespace {

constexpr int RB_T = 256;
constexpr int RB_FRAC = 48;

struct RBParams {
  int32_t n;
  int32_t Tc;                 // trees in this chunk
  const int64_t* rowptr;
  const int32_t* colidx;
  const float* w;             // or null
  double alpha;
  const double* alpha_v;      // per-vertex alpha (batches) or null
  const int32_t* parents;     // [Tc][n]
  uint64_t* acc;              // [n] fixed-point sums
  // scratch, flat index i = t * n + v
  uint32_t* cnt;              // children counts
  uint32_t* off;              // exclusive prefix of cnt (flat)
  int32_t* child;             // children of every (tree, vertex), contiguous
  int32_t* ordr;              // flat ids level by level (BFS order)
  int32_t* lvl;               // [n + 2] level offsets into ordr
  int32_t* size;              // fill counter during the scatter, then subtree sizes
  int32_t* tin;               // preorder numbers
  uint32_t* bsum;             // [gridDim.x] block totals of the scan
  uint32_t* ctr;              // [0] ordr appends, [2] error
  uint32_t* next_tin;         // [Tc] next free preorder number per tree
};

__device__ __forceinline__ uint32_t block_exscan_u32(uint32_t x, uint32_t* total, uint32_t* wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t s = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += y;
  }
  if (lane == 31) wsum[wid] = s;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  const uint32_t ex = s - x + (wid > 0 ? wsum[wid - 1] : 0u);
  *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return ex;
}

__global__ void __launch_bounds__(RB_T) k_rb(RBParams p) {
  cg::grid_group grid = cg::this_grid();
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t sh_carry;
  const int32_t n = p.n;
  const int64_t N = (int64_t)p.Tc * n;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;

  // ---- child counts; parents must lie in [0, n] and differ from the vertex ----
  for (int64_t i = gtid; i < N; i += gstride) {
    const int32_t v = (int32_t)(i % n);
    const int32_t par = p.parents[i];
    p.size[i] = 0;
    if (par < 0 || par > n || par == v) atomicOr(&p.ctr[2], ERR_INVAL);
    else if (par < n) atomicAdd(&p.cnt[i - v + par], 1u);
  }
  grid.sync();
  if (*(volatile uint32_t*)&p.ctr[2] != 0u) return;  // uniform: read after the barrier

  // ---- exclusive scan of cnt over the flat index: block ranges, then block totals ----
  const int64_t chunk = (N + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = std::min<int64_t>(N, b0 + chunk);
  if (threadIdx.x == 0) sh_carry = 0;
  __syncthreads();
  for (int64_t base = b0; base < b1; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const uint32_t x = i < b1 ? p.cnt[i] : 0u;
    uint32_t tot = 0;
    const uint32_t ex = block_exscan_u32(x, &tot, wsum);
    if (i < b1) p.off[i] = sh_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) sh_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) p.bsum[blockIdx.x] = sh_carry;
  grid.sync();
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) sh_carry = 0;
    __syncthreads();
    for (int base = 0; base < (int)gridDim.x; base += blockDim.x) {
      const int j = base + threadIdx.x;
      const uint32_t x = j < (int)gridDim.x ? p.bsum[j] : 0u;
      uint32_t tot = 0;
      const uint32_t ex = block_exscan_u32(x, &tot, wsum);
      if (j < (int)gridDim.x) p.bsum[j] = sh_carry + ex;
      __syncthreads();
      if (threadIdx.x == 0) sh_carry += tot;
      __syncthreads();
    }
  }
  grid.sync();
  {
    const uint32_t add = p.bsum[blockIdx.x];
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) p.off[i] += add;
  }
  grid.sync();

  // ---- children (in any order) and the roots as BFS level 0 ----
  for (int64_t i = gtid; i < N; i += gstride) {
    const int32_t v = (int32_t)(i % n);
    const int32_t par = p.parents[i];
    if (par < n) {
      const int64_t pi = i - v + par;
      p.child[p.off[pi] + (uint32_t)atomicAdd(&p.size[pi], 1)] = v;
    } else {
      p.ordr[atomicAdd(&p.ctr[0], 1u)] = (int32_t)i;
    }
  }
  grid.sync();
  if (gtid == 0) {
    p.lvl[0] = 0;
    p.lvl[1] = (int32_t)p.ctr[0];
  }
  grid.sync();

  // ---- BFS levels: level d is ordr[lvl[d], lvl[d + 1]) ----
  int32_t D = 0;  // levels
  for (int32_t d = 0; d <= n; ++d) {
    const int32_t a0 = *(volatile int32_t*)&p.lvl[d], a1 = *(volatile int32_t*)&p.lvl[d + 1];
    if (a1 == a0) {
      D = d;
      break;
    }
    for (int64_t j = a0 + gtid; j < a1; j += gstride) {
      const int32_t i = p.ordr[j];
      const int32_t t0 = i - i % n;
      const uint32_t c0 = p.off[i], cn = p.cnt[i];
      for (uint32_t k = 0; k < cn; ++k) p.ordr[atomicAdd(&p.ctr[0], 1u)] = t0 + p.child[c0 + k];
    }
    grid.sync();
    if (gtid == 0) p.lvl[d + 2] = (int32_t)p.ctr[0];
    grid.sync();
  }
  if (*(volatile int32_t*)&p.lvl[D] != (int32_t)N) {  // a parent cycle: not a forest rooted at u*
    if (gtid == 0) atomicOr(&p.ctr[2], ERR_INVAL);
    return;  // uniform: every CTA read the same lvl[D]
  }

  // ---- subtree sizes, deepest level first ----
  for (int32_t d = D - 1; d >= 0; --d) {
    const int32_t a0 = p.lvl[d], a1 = p.lvl[d + 1];
    for (int64_t j = a0 + gtid; j < a1; j += gstride) {
      const int32_t i = p.ordr[j];
      const int32_t t0 = i - i % n;
      const uint32_t c0 = p.off[i], cn = p.cnt[i];
      int32_t s = 1;
      for (uint32_t k = 0; k < cn; ++k) s += p.size[t0 + p.child[c0 + k]];
      p.size[i] = s;
    }
    grid.sync();
  }

  // ---- preorder numbers, roots first, then each vertex numbers its children ----
  for (int64_t j = gtid; j < p.lvl[1]; j += gstride) {
    const int32_t i = p.ordr[j];
    p.tin[i] = (int32_t)atomicAdd(&p.next_tin[i / n], (uint32_t)p.size[i]);
  }
  grid.sync();
  for (int32_t d = 0; d + 1 < D; ++d) {
    const int32_t a0 = p.lvl[d], a1 = p.lvl[d + 1];
    for (int64_t j = a0 + gtid; j < a1; j += gstride) {
      const int32_t i = p.ordr[j];
      const int32_t t0 = i - i % n;
      const uint32_t c0 = p.off[i], cn = p.cnt[i];
      int32_t run = p.tin[i] + 1;
      for (uint32_t k = 0; k < cn; ++k) {
        const int32_t ci = t0 + p.child[c0 + k];
        p.tin[ci] = run;
        run += p.size[ci];
      }
    }
    grid.sync();
  }

  // ---- the conditional probability of every (tree, vertex) ----
  for (int64_t i = gtid; i < N; i += gstride) {
    const int32_t v = (int32_t)(i % n);
    const int64_t t0 = i - v;
    const int32_t lo = p.tin[i], hi = lo + p.size[i];
    double s = 0.0;
    for (int64_t e = p.rowptr[v]; e < p.rowptr[v + 1]; ++e) {
      const int32_t tu = p.tin[t0 + p.colidx[e]];
      if (tu < lo || tu >= hi) s = __dadd_rn(s, p.w ? (double)p.w[e] : 1.0);
    }
    const double a = p.alpha_v ? p.alpha_v[v] : p.alpha;
    const double val = __ddiv_rn(1.0, __dadd_rn(1.0, __dmul_rn(a, s)));
    const uint64_t q = (uint64_t)__dadd_rn(__dmul_rn(val, (double)(1ull << RB_FRAC)), 0.5);
    atomicAdd((unsigned long long*)&p.acc[v], (unsigned long long)q);
  }
}

__global__ void k_rb_diag(int32_t n, const uint64_t* __restrict__ acc, double denom, double* __restrict__ diag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    diag[v] = __ddiv_rn((double)acc[v], denom);
}

}  // namespace

}  // namespace fcx

using namespace fcx;

extern "C" fc_status fc_rb_accumulate(fc_graph* g, int32_t alpha_idx, const int32_t* parents, int64_t T,
                                      uint64_t* acc, void* stream) {
  if (g == nullptr || parents == nullptr || acc == nullptr || T < 0 || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha) {
    set_error("fc_rb_accumulate: bad argument");
    return FC_EINVAL;
  }
  if (T == 0) return FC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  int dev = g->device, nsm = 0, coop = 0, per_sm = 0;
  FC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FC_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) {
    set_error("fc_rb_accumulate: the device does not support cooperative launches");
    return FC_ECUDA;
  }
  FC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rb, RB_T, 0));
  const int grid = std::max(1, per_sm) * nsm;  // every CTA resident: required by the grid barriers
  // trees per chunk: 24 bytes of scratch per (tree, vertex), at most 4 GB and
  // flat ids below 2^31
  const int64_t cap = std::max<int64_t>(1, std::min<int64_t>((int64_t)(4ull << 30) / (24ll * n),
                                                             ((int64_t)1 << 31) / ((int64_t)n + 1) - 1));
  const int64_t Tc_max = std::min<int64_t>(T, cap);
  const size_t N = (size_t)Tc_max * n;
  char* ws = nullptr;
  const size_t bytes = N * 4 * 6 + ((size_t)n + 2) * 4 + (size_t)grid * 4 + 16 + (size_t)Tc_max * 4 + 256 * 8;
  FC_CK(cudaMallocAsync((void**)&ws, bytes, st));
  auto carve = [&](size_t b) {
    char* r = ws;
    ws += (b + 255) & ~(size_t)255;
    return r;
  };
  char* base = ws;
  RBParams p;
  p.n = n;
  p.rowptr = g->rowptr;
  p.colidx = g->colidx;
  p.w = g->w;
  p.alpha = g->alphas[alpha_idx];
  p.alpha_v = g->num_graphs > 0 ? g->alpha_v : nullptr;
  p.acc = acc;
  p.cnt = (uint32_t*)carve(N * 4);
  p.off = (uint32_t*)carve(N * 4);
  p.child = (int32_t*)carve(N * 4);
  p.ordr = (int32_t*)carve(N * 4);
  p.size = (int32_t*)carve(N * 4);
  p.tin = (int32_t*)carve(N * 4);
  p.lvl = (int32_t*)carve(((size_t)n + 2) * 4);
  p.bsum = (uint32_t*)carve((size_t)grid * 4);
  p.ctr = (uint32_t*)carve(16);
  p.next_tin = (uint32_t*)carve((size_t)Tc_max * 4);
  ws = base;
  fc_status status = FC_OK;
  for (int64_t t0 = 0; t0 < T && status == FC_OK; t0 += Tc_max) {
    const int32_t Tc = (int32_t)std::min<int64_t>(Tc_max, T - t0);
    p.Tc = Tc;
    p.parents = parents + (size_t)t0 * n;
    const size_t Nc = (size_t)Tc * n;
    FC_CK(cudaMemsetAsync(p.cnt, 0, Nc * 4, st));
    FC_CK(cudaMemsetAsync(p.ctr, 0, 16, st));
    FC_CK(cudaMemsetAsync(p.next_tin, 0, (size_t)Tc * 4, st));
    void* args[] = {&p};
    FC_CK(cudaLaunchCooperativeKernel((void*)k_rb, dim3(grid), dim3(RB_T), args, 0, st));
    FC_LAUNCHED();
    uint32_t herr = 0;
    FC_CK(cudaMemcpyAsync(&herr, p.ctr + 2, 4, cudaMemcpyDeviceToHost, st));
    FC_CK(cudaStreamSynchronize(st));
    if (herr != 0) {
      set_error("fc_rb_accumulate: parents do not form spanning trees of G* rooted at u* = n");
      status = FC_EINVAL;
    }
  }
  FC_CK(cudaFreeAsync(base, st));
  return status;
}

extern "C" fc_status fc_rb_diag(const uint64_t* acc, int32_t n, int64_t T, double* diag_out, void* stream) {
  if (acc == nullptr || diag_out == nullptr || n < 1 || T < 1) {
    set_error("fc_rb_diag: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const double denom = (double)(1ull << RB_FRAC) * (double)T;  // exact: a power of two times T
  k_rb_diag<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(n, acc, denom, diag_out);
  FC_LAUNCHED();
  return FC_OK;
}
