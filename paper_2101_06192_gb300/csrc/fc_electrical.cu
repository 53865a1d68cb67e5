// Electrical closeness on G (Sec. 3: the diag(L^+) algorithm that the forest
// algorithm builds on, insights (i)-(iii); Eq. 2; Def. 2 with the effective
// resistance in place of the forest distance).
//
//   fc_build_rooted           G with walks whose only exit is the pivot u, and
//                             u's breadth-first tree B (the fixed paths of the
//                             resistance estimator); rejects disconnected G
//   fc_sample_usts            (fc_wilson*.cu) uniform spanning trees of G rooted at u
//   fc_resistance_accumulate  (fc_rb.cu) Kirchhoff path sums along B
//   fc_laplacian_solve        (fc_solve.cu) the pivot column x = L^+ e_u
//   fc_electrical_closeness   r^(u, v) from the path sums or from the sampler's
//                             visit totals (Green's function), L^+[v, v] = r^ -
//                             x[u] + 2 x[v] (Eq. 2), farness n L^+[v, v] +
//                             tr(L^+), closeness n / farness
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "fc_internal.cuh"

namespace cg = cooperative_groups;

namespace fcx {

namespace {

constexpr int BFS_T = 256;
constexpr int EL_T = 256;
constexpr int EL_FRAC = 32;  // fixed-point fraction bits of the path-sum totals

// Breadth-first levels from the root, one cooperative launch, into one
// queue holding the levels one after another (queue[0] = root): level L is
// queue[base, base + len) with len in counter L % 3; its new vertices are
// appended after it through counter (L + 1) % 3; counter (L + 2) % 3, last
// read at level L - 1, is cleared for level L + 1.  depth[] starts at -1
// (host memset) with the root at 0; a vertex joins the level that first
// claims it.  The queue is a breadth-first order of the vertices.
__global__ void __launch_bounds__(BFS_T) k_bfs(int32_t n, const int64_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ colidx, int32_t root,
                                               int32_t* __restrict__ depth, int32_t* __restrict__ queue,
                                               uint32_t* __restrict__ counters) {
  cg::grid_group grid = cg::this_grid();
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  for (int32_t level = 0;; ++level) {
    const uint32_t len = *(volatile uint32_t*)&counters[level % 3];
    if (len == 0u) break;  // uniform: read after the barrier that ended the last level
    if (gtid == 0) counters[(level + 2) % 3] = 0u;
    int32_t* nxt = queue + base + len;
    // a warp per frontier vertex, its lanes over the row
    for (int64_t i = gtid >> 5; i < (int64_t)len; i += gstride >> 5) {
      const int32_t x = queue[base + i];
      for (int64_t e = rowptr[x] + lane; e < rowptr[x + 1]; e += 32) {
        const int32_t y = colidx[e];
        if (atomicCAS(&depth[y], -1, level + 1) == -1) nxt[atomicAdd(&counters[(level + 1) % 3], 1u)] = y;
      }
    }
    if (gtid == 0) atomicMax(&counters[3], (uint32_t)level);
    grid.sync();
    base += len;
  }
}

// The parent of v in the breadth-first tree: its smallest-id neighbour one
// level closer to the root (a warp per vertex), and 1 / w of that edge in
// FP64.  Counts unreached vertices in *unreached.
__global__ void k_bfs_parent(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                             const float* __restrict__ w, const int32_t* __restrict__ depth, int32_t root,
                             int32_t* __restrict__ bpar, double* __restrict__ binv, uint32_t* __restrict__ unreached) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t dv = depth[v];
    if (v == root || dv < 0) {
      if (lane == 0) {
        bpar[v] = -1;
        binv[v] = 0.0;
        if (dv < 0) atomicAdd(unreached, 1u);
      }
      continue;
    }
    int32_t best = INT32_MAX;
    int64_t best_e = -1;
    for (int64_t e = rowptr[v] + lane; e < rowptr[v + 1]; e += 32) {
      const int32_t y = colidx[e];
      if (depth[y] == dv - 1 && y < best) {
        best = y;
        best_e = e;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t oe = __shfl_xor_sync(0xffffffffu, best_e, o);
      if (ob < best) {
        best = ob;
        best_e = oe;
      }
    }
    if (lane == 0) {
      bpar[v] = best;
      binv[v] = w ? __ddiv_rn(1.0, (double)w[best_e]) : 1.0;
    }
  }
}

// r^(root, v) from the path-sum totals, acc[v] / (2^32 T), or from the visit
// totals, visits[v] / (T d_w(v)) (0 at the root); then d_v = r^ - x[root] +
// 2 x[v] (Eq. 2 solved for L^+[v, v]) and per-block partial sums of d
// (fixed-order tree).
__global__ void k_el_combine(int32_t n, const int64_t* __restrict__ acc, const unsigned long long* __restrict__ visits,
                             const double* __restrict__ dw, double trees, double denom,
                             const double* __restrict__ x, int32_t root, double* __restrict__ resist,
                             double* __restrict__ diag, double* __restrict__ partial) {
  __shared__ double red[EL_T];
  const int64_t v = (int64_t)blockIdx.x * EL_T + threadIdx.x;
  double d = 0.0;
  if (v < n) {
    const double r = acc ? __ddiv_rn((double)acc[v], denom)
                         : (v == root ? 0.0 : __ddiv_rn((double)visits[v], __dmul_rn(trees, dw[v])));
    d = __dadd_rn(__dadd_rn(r, -x[root]), __dmul_rn(2.0, x[v]));
    if (resist) resist[v] = r;
    diag[v] = d;
  }
  red[threadIdx.x] = d;
  __syncthreads();
  for (int s = EL_T / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_el_sum(const double* __restrict__ partial, int64_t m, double* __restrict__ out) {
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

// farness = n L^+[v, v] + tr(L^+) (the sum of Eq. 2 over v); closeness n / farness
__global__ void k_el_farness(int32_t n, const double* __restrict__ diag, const double* __restrict__ trace,
                             double* __restrict__ farness, double* __restrict__ closeness) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double f = (double)n * diag[v] + *trace;
  if (farness) farness[v] = f;
  if (closeness) closeness[v] = (double)n / f;
}

}  // namespace

}  // namespace fcx

using namespace fcx;

extern "C" fc_status fc_build_rooted(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                     const float* w, int32_t root, uint32_t flags, void* stream, fc_graph** out) {
  if (out == nullptr) {
    set_error("fc_build_rooted: null output pointer");
    return FC_EINVAL;
  }
  *out = nullptr;
  if (n < 2 || root < 0 || root >= n) {
    set_error("fc_build_rooted: need n >= 2 and 0 <= root < n");
    return FC_EINVAL;
  }
  const double one = 1.0;
  fc_graph* g = nullptr;
  const fc_status s = build_impl(n, nnz, rowptr, colidx, w, &one, 1, flags, stream, &g, 0, nullptr, nullptr, root);
  if (s != FC_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* qa = nullptr;
  uint32_t* ctr = nullptr;
  auto fail = [&](fc_status code) {
    if (qa) cudaFreeAsync(qa, st);
    if (ctr) cudaFreeAsync(ctr, st);
    cudaStreamSynchronize(st);
    fc_destroy(g);
    return code;
  };
  cudaError_t e = cudaMallocAsync((void**)&g->bpar, (size_t)n * sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&g->binv, (size_t)n * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&g->bdepth, (size_t)n * sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&qa, (size_t)n * sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&ctr, 8 * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->bdepth, 0xff, (size_t)n * sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->bdepth + root, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(qa, &root, sizeof(int32_t), cudaMemcpyHostToDevice, st);
  const uint32_t c0[8] = {1u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};  // frontier 0 = {root}; [3] deepest level; [4] unreached
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctr, c0, sizeof(c0), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(cuda_fail(e, "fc_build_rooted: breadth-first tree scratch"));
  int nsm = 0, per_sm = 0, coop = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs, BFS_T, 0);
  if (e != cudaSuccess) return fail(cuda_fail(e, "fc_build_rooted: device attributes"));
  if (!coop) {
    set_error("fc_build_rooted: the device does not support cooperative launches");
    return fail(FC_ECUDA);
  }
  {
    void* args[] = {&n, &g->rowptr, &g->colidx, &root, &g->bdepth, &qa, &ctr};
    e = cudaLaunchCooperativeKernel((void*)k_bfs, dim3(std::max(1, per_sm) * nsm), dim3(BFS_T), args, 0, st);
    fcx::note_launch();
    if (e != cudaSuccess) return fail(cuda_fail(e, "fc_build_rooted: k_bfs"));
  }
  k_bfs_parent<<<(unsigned)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, (int64_t)nsm * 64), 256, 0, st>>>(
      n, g->rowptr, g->colidx, g->w, g->bdepth, root, g->bpar, g->binv, ctr + 4);
  fcx::note_launch();
  e = cudaGetLastError();
  uint32_t hc[8] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_fail(e, "fc_build_rooted: breadth-first tree"));
  if (hc[4] != 0u) {
    set_error("fc_build_rooted: G is not connected (electrical closeness is defined on connected graphs)");
    return fail(FC_EINVAL);
  }
  g->max_bdepth = (int32_t)hc[3];
  // Start vertices in the reverse of the breadth-first order (the farthest
  // first).  Measured on GB300 (BA n = 2^20 rooted at its hub, 256 trees,
  // 1024 walkers): 372 ms against 453 ms in breadth-first order and 615 ms in
  // vertex-id order.  The trees do not depend on the order.
  e = cudaMemcpyAsync(g->order, qa, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fail(cuda_fail(e, "fc_build_rooted: start order"));
  g->order_auto = false;
  g->order_id = 0;
  g->order_desc = 1;
  cudaFreeAsync(qa, st);
  cudaFreeAsync(ctr, st);
  cudaStreamSynchronize(st);
  *out = g;
  return FC_OK;
}

extern "C" fc_status fc_bfs_tree(const fc_graph* g, int32_t* parent_out, int32_t* depth_out, void* stream) {
  if (g == nullptr || g->root < 0 || g->bpar == nullptr) {
    set_error("fc_bfs_tree: needs a graph from fc_build_rooted");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (parent_out)
    FC_CK(cudaMemcpyAsync(parent_out, g->bpar, (size_t)g->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  if (depth_out)
    FC_CK(cudaMemcpyAsync(depth_out, g->bdepth, (size_t)g->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return FC_OK;
}

extern "C" fc_status fc_electrical_closeness(fc_graph* g, const int64_t* acc, const uint64_t* visits, int64_t T,
                                             const double* x_pivot, double* resist_out, double* diag_out,
                                             double* farness_out, double* closeness_out, void* stream) {
  if (g == nullptr || (acc == nullptr) == (visits == nullptr) || x_pivot == nullptr || diag_out == nullptr ||
      T < 1) {
    set_error("fc_electrical_closeness: bad argument");
    return FC_EINVAL;
  }
  if (g->root < 0) {
    set_error("fc_electrical_closeness: needs a graph from fc_build_rooted");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  const int64_t nb = (n + EL_T - 1) / EL_T;
  double* part = nullptr;
  FC_CK(cudaMallocAsync((void**)&part, (size_t)(nb + 1) * sizeof(double), st));
  const double denom = (double)(1ull << EL_FRAC) * (double)T;  // exact: a power of two times T < 2^53
  k_el_combine<<<(unsigned)nb, EL_T, 0, st>>>(n, acc, (const unsigned long long*)visits, g->dw, (double)T, denom,
                                              x_pivot, g->root, resist_out, diag_out, part);
  FC_LAUNCHED();
  k_el_sum<<<1, 1024, 0, st>>>(part, nb, part + nb);
  FC_LAUNCHED();
  if (farness_out || closeness_out) {
    k_el_farness<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, diag_out, part + nb, farness_out, closeness_out);
    FC_LAUNCHED();
  }
  FC_CK(cudaFreeAsync(part, st));
  return FC_OK;
}
