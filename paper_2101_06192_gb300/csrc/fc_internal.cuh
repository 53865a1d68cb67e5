// Internal definitions shared by the fc CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "fc.h"

namespace fcx {

// ---------------------------------------------------------------------------
// Error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
fc_status cuda_fail(cudaError_t e, const char* what);

#define FC_CK(call)                                      \
  do {                                                   \
    cudaError_t fc_e_ = (call);                          \
    if (fc_e_ != cudaSuccess) return fcx::cuda_fail(fc_e_, #call); \
  } while (0)

// Every kernel launch of the library is followed by FC_LAUNCHED(): it counts
// the launch (fc_launch_count) and checks the launch error.
void note_launch();
#define FC_LAUNCHED()                                    \
  do {                                                   \
    fcx::note_launch();                                  \
    FC_CK(cudaGetLastError());                           \
  } while (0)

// Process-wide device scratch for the sampler's per-tree state: grown on
// demand, reused across graphs and calls, released by fc_release_scratch.
fc_status sampler_scratch(int device, size_t bytes, cudaStream_t st, void** out, bool capturing = false);

// Graph construction shared by fc_build_augmented, fc_build_batch and
// fc_build_rooted (root >= 0: walks on G whose only exit is that vertex).
fc_status build_impl(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx, const float* w,
                     const double* alphas, int32_t n_alpha, uint32_t flags, void* stream, fc_graph** out, int32_t G,
                     const int64_t* voff_h, const double* galpha_h, int32_t root);
void free_graph_arrays(fc_graph* g, cudaStream_t st);

// Keep freed stream-ordered allocations in the device's default pool.
void retain_pool(int device);

// Exclusive prefix sum of len uint32 values on `st` (multi-level, temporary
// memory from the stream-ordered pool).
fc_status exclusive_scan(const uint32_t* in, uint32_t* out, int64_t len, cudaStream_t st);

// Device error word bits (OR-ed by kernels, read back by the host).
enum : uint32_t {
  ERR_INVAL = 1u,
  ERR_TIMEOUT = 2u,
  ERR_OVERFLOW = 4u,
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): 10 rounds of the 4x32 S-box with multipliers
// 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// 53 uniform bits of one stack entry (words 0 and 1).
__device__ __forceinline__ uint64_t stack_u53(const uint4& o) {
  return ((uint64_t)o.x << 21) | (uint64_t)(o.y >> 11);
}

// ---------------------------------------------------------------------------
// Exact integer thresholds of the FP64 selector.
//   x(u) = fl(fl(u * 2^-53) * t), clamped to the largest double below t.
//   count_below(c, t) = #{u in [0, 2^53) : x(u) < c}.
// x is monotone in u, so {u : x(u) < c} is a prefix [0, count).  All FP ops are
// explicit _rn intrinsics: no contraction, identical to the IEEE sequence.
// ---------------------------------------------------------------------------
constexpr uint64_t TWO53 = 1ull << 53;

__host__ __device__ __forceinline__ double below_pos(double t) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(__double_as_longlong(t) - 1);
#else
  long long b;
  memcpy(&b, &t, sizeof(b));
  b -= 1;
  double r;
  memcpy(&r, &b, sizeof(r));
  return r;
#endif
}

__device__ __forceinline__ double sel_x(uint64_t u, double t) {
  const double U = __dmul_rn((double)u, 0x1.0p-53);
  double x = __dmul_rn(U, t);
  if (x >= t) x = below_pos(t);
  return x;
}

__device__ inline uint64_t count_below(double c, double t) {
  if (!(c > 0.0)) return 0;
  if (c >= t) return TWO53;  // x(u) < t for every u (clamp)
  double q = __dmul_rn(__ddiv_rn(c, t), 0x1.0p53);
  uint64_t u = q <= 0.0 ? 0ull : (q >= 0x1.0p53 ? TWO53 : (uint64_t)q);
  // smallest u with x(u) >= c; the estimate is within a few units
  for (int it = 0; it < 4096; ++it) {
    if (u > 0 && sel_x(u - 1, t) >= c) { --u; continue; }
    if (u < TWO53 && sel_x(u, t) < c) { ++u; continue; }
    return u;
  }
  // fallback: bisection over [0, 2^53]
  uint64_t lo = 0, hi = TWO53;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (sel_x(mid, t) < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// t = fl(1 + fl(alpha * s))
__device__ __forceinline__ double deg_star(double alpha, double s) {
  return __dadd_rn(1.0, __dmul_rn(alpha, s));
}

// t = fl(gamma + fl(alpha * s)): gamma = 1 on G* (the u* edge), 0 for walks
// on G itself (fl(0 + s) = s exactly)
__device__ __forceinline__ double deg_gamma(double gamma, double alpha, double s) {
  return __dadd_rn(gamma, __dmul_rn(alpha, s));
}

}  // namespace fcx

// ---------------------------------------------------------------------------
// The graph object behind the opaque fc_graph handle.
// ---------------------------------------------------------------------------
struct fc_graph {
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t n_alpha = 0;
  bool weighted = false;
  int device = 0;
  size_t device_bytes = 0;  // total device memory, read at build
  std::vector<double> alphas;
  // device arrays owned by the graph
  int64_t* rowptr = nullptr;   // [n+1]
  int32_t* colidx = nullptr;   // [nnz]
  float* w = nullptr;          // [nnz] or null
  int32_t* deg = nullptr;      // [n]
  double* dw = nullptr;        // [n] weighted degree (FP64, left-to-right per row)
  double* S = nullptr;         // [nnz] per-row FP64 prefix of w (weighted only)
  int32_t* order = nullptr;    // [n] ascending degree, ties by id
  uint4* rowinfo = nullptr;    // [n_alpha][n] {row offset, degree, T lo, T hi}
  uint64_t* B = nullptr;       // [n_alpha][nnz] slot thresholds (weighted only)
  uint4* edges = nullptr;      // [n_alpha][nnz] edge records (single graphs; 64 bytes when weighted)
  double* alphas_d = nullptr;  // [n_alpha]
  int32_t max_deg = 0;
  // G rooted at a pivot vertex (fc_build_rooted; -1 for G*): walks on G whose
  // only exit is the pivot, and the pivot's breadth-first tree
  int32_t root = -1;
  int32_t* bpar = nullptr;     // [n] BFS parent (-1 at the root)
  double* binv = nullptr;      // [n] 1 / w(v, bpar(v)) in FP64 (0 at the root)
  int32_t* bdepth = nullptr;   // [n] BFS depth
  int32_t max_bdepth = 0;
  // batch of graphs (block-diagonal union with one alpha per graph)
  int32_t num_graphs = 0;      // 0 = a single graph
  int64_t* voff = nullptr;     // [G+1] vertex offsets
  int32_t* gid = nullptr;      // [n] graph of each vertex
  double* alpha_v = nullptr;   // [n] alpha of each vertex's graph
  int32_t* gorder = nullptr;   // [G] graphs by decreasing size (work order)
  int32_t max_ng = 0;          // largest graph
  std::vector<int64_t> voff_h;
  std::vector<double> galpha;
  unsigned long long* item_ns = nullptr;  // [G * tau_last] completion times of the last launch
  size_t item_cap = 0;
  int64_t last_tau = 0;
  unsigned long long* t0_ns = nullptr;    // earliest CTA start of the last launch
  // sampler shape
  int32_t walkers = 0;
  int32_t max_trees = 0;
  int32_t smem_mode = 0;
  int32_t regs = 0;            // register cap of the sampler variant (0 = automatic)
  int32_t order_desc = 0;      // sampler takes start vertices from the high end of the order
  int32_t order_id = 0;        // start order: 0 = degree, 1 = vertex id (fc_set_start_order)
  bool order_auto = true;      // automatic start order (the default): vertex id unless id_local
  bool id_local = false;       // the vertex numbering follows the graph's geometry (build-time statistic)
  int32_t kernel_pref = 0;     // 0 = automatic, 1 = CSR-walk kernel, 2 = edge-record kernel
  int32_t pops_mode = 0;       // 0 = automatic, 1 = walk every cycle, 2 = pop from the ring (fc_set_sampler_pops)
  int32_t bitmap_mode = 0;     // 0 = automatic, 1 = state flags, 2 = shared, 3 = global (fc_set_sampler_bitmap)
  int32_t cluster = 0;         // CTAs per tree of the edge-record kernel (0 = automatic; fc_set_sampler_cluster)
  int32_t last_cluster = 0;    // CTAs per tree of the last launch
  int32_t last_kernel = 0;     // kernel of the last launch (1 or 2)
  int32_t last_W = 0, last_regs = 0, last_grid = 0;  // shape of the last launch
  // results of the launch-shape search for the last SHAPE_SLOTS distinct inputs
  // (launches of a few alternating tree counts, such as a run that samples up
  // to increasing checkpoints, reuse them), replaced round-robin
  static constexpr int SHAPE_SLOTS = 8;
  int64_t shape_key[SHAPE_SLOTS][12] = {};
  int64_t shape_val[SHAPE_SLOTS][6] = {};
  bool shape_used[SHAPE_SLOTS] = {};
  int32_t shape_next = 0;
  // scratch owned by the graph
  void* ws = nullptr;          // sampler per-tree state
  size_t ws_bytes = 0;
  uint32_t* d_err = nullptr;   // device error word
  unsigned long long* d_counter = nullptr;  // sampler work queue
  unsigned long long* d_stats = nullptr;    // [2] pops, departures of the last launch
  // solver scratch
  void* sv = nullptr;
  size_t sv_bytes = 0;
};
