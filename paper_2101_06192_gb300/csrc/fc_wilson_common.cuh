// Definitions shared by the two Wilson sampler kernels (the CSR-walk kernel
// and the edge-record kernel): per-vertex tree state, launch parameters, the
// stack-entry slot decision and L2-policy memory operations.
#pragma once

#include "fc_internal.cuh"

namespace fcx {

struct __align__(16) VState {
  unsigned long long st;
  uint32_t nxt;
  uint32_t pad;
};

constexpr int K_BITS = 24;
constexpr unsigned long long K_MASK = (1ull << K_BITS) - 1;
constexpr int W_BITS = 10;
constexpr unsigned FULL = 0xffffffffu;

struct WParams {
  int32_t n;
  int32_t n_alpha;
  int64_t nnz;
  const uint4* rowinfo;     // [n_alpha][n] {row offset, degree, T lo, T hi}
  const int32_t* colidx;    // [nnz]
  const int32_t* order;     // [n] start order (ascending degree)
  const uint64_t* B;        // [n_alpha][nnz] slot thresholds, or null (unweighted)
  int64_t tau;
  int64_t tree_offset;
  uint32_t key0, key1;
  uint32_t* R;              // [n_alpha][n]
  uint32_t* C;              // [n_alpha][n] or null
  int32_t* parents;         // [n_alpha*tau][n] or null
  uint64_t* steps;          // [n_alpha*tau] or null
  unsigned long long* visits;  // [n_alpha][n]: += departures from each vertex per tree, or null
  VState* gstate;           // [gridDim.x][n] (global-state variant)
  uint32_t* gbits;          // [gridDim.x][words] in-tree bitmaps (global-state variant)
  int32_t words;            // bitmap words per tree: ceil(nmax / 32)
  int32_t nmax;             // vertices of the largest tree of the launch (state records per CTA)
  int pre_cleared;          // the first tree of every CTA starts from host-cleared state
  unsigned long long* counter;
  uint32_t* err;
  unsigned long long* stats;  // [0] pops, [1] departures, [2..] iteration counters (N_CNT)
  uint32_t max_iters;
  int descending;           // take start vertices from the high-degree end (or the high-id end)
  int id_order;             // start vertices in vertex-id order instead of the degree order
  const uint4* edges;       // [n_alpha][nnz] edge records {target, its row offset, its degree,
                            //  its threshold >> 21} (edge-record kernel; weighted graphs: 64-byte
                            //  records, the header followed by 12 slot-threshold high words)
  // batch of graphs: work item i samples tree (i % tau) of graph gorder[i / tau]
  int32_t num_graphs;       // 0 = single graph
  const int64_t* voff;      // [G+1]
  const int32_t* gorder;    // [G] graphs by decreasing size
  unsigned long long* item_ns;  // [G*tau] %globaltimer at completion, indexed graph-major (or null)
  unsigned long long* t0_ns;    // earliest CTA start (or null)
  // edge-record kernel without clusters: warp w of a CTA takes start vertices
  // only once its tree holds at least w * ramp_q vertices (or every start
  // position is handed out); 0 = every warp from the start
  uint32_t ramp_q;
  // forest roots and depths ([rows][n] like parents, either may be null;
  // edge-record kernel without clusters): each vertex's {root, depth} is put
  // in rdpack ([gridDim.x][nmax], 8 bytes) when it joins the tree and copied
  // out by the end-of-tree pass
  int32_t* roots;
  int32_t* depths;
  unsigned long long* rdpack;
};

// Pop and release walks read a vertex's nxt, then free the vertex with an
// atomic on its state word.  The two are different fields, so neither the
// compiler nor the memory system has to keep that order, and a vertex freed
// first can be claimed by another walker, which rewrites its nxt before the
// read.  Freeing under a test of the loaded value (never all ones: nxt holds a
// vertex id or n) makes the atomic wait for the load.
__device__ __forceinline__ bool nxt_read(uint32_t nc) { return nc != 0xffffffffu; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Iteration counters (diagnostic), summed over walkers and trees.
enum { CNT_ITER = 0, CNT_CLAIM_OK, CNT_TREE_HIT, CNT_CONFIRM, CNT_SPIN, CNT_WAIT, CNT_RELEASE, CNT_POP,
       CNT_EDGE, CNT_IDLE_LANE, N_CNT };

// Slot decision for one stack entry with Philox words o at a vertex with row
// info ri = {row offset, degree, T lo, T hi}: returns true and sets *edge to
// the CSR entry of the selected neighbour, or false when the entry selects u*
// (u53 < T).  The neighbour is floor(o2 d / 2^32) (unweighted) or the first
// entry of the row with u53 < B (weighted; the last B of a row is 2^53).
__device__ __forceinline__ bool select_edge(const WParams& p, int a, const uint4& ri, const uint4& o,
                                            uint32_t* edge) {
  const uint32_t d = ri.y;
  const uint64_t u = stack_u53(o);
  const uint64_t T = (uint64_t)ri.z | ((uint64_t)ri.w << 32);
  if (u < T) return false;
  if (p.B == nullptr) {
    *edge = ri.x + __umulhi(o.z, d);
    return true;
  }
  const uint64_t* b = p.B + (size_t)a * p.nnz + ri.x;
  uint32_t lo = 0, hi = d - 1;
  if (d <= 8) {
    // short rows: all thresholds in flight at once
    uint64_t bv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) bv[j] = (j < (int)d - 1) ? __ldg(b + j) : ~0ull;
#pragma unroll
    for (int j = 7; j >= 0; --j)
      if (u < bv[j]) lo = (uint32_t)j;
    lo = min(lo, d - 1);
  } else {
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (u < __ldg(b + mid)) hi = mid; else lo = mid + 1;
    }
  }
  *edge = ri.x + lo;
  return true;
}

constexpr int PB = 8;  // path vertices remembered per walker (shared memory)

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* a) {
  return *(const volatile unsigned long long*)a;
}
__device__ __forceinline__ uint32_t ld_volatile32(const uint32_t* a) {
  return *(const volatile uint32_t*)a;
}

// Per-iteration diagnostic counters (fc_sampler_counters) are compiled in only
// with -DFC_WILSON_COUNTERS=1; they cost registers in the walk loop.
#ifndef FC_WILSON_COUNTERS
#define FC_WILSON_COUNTERS 0
#endif
#if FC_WILSON_COUNTERS
#define CNT(q) (++cnt[q])
#else
#define CNT(q) ((void)0)
#endif

typedef void (*WilsonFn)(WParams);

// Edge-record kernel (single graphs, state in global memory) with tree
// membership as flags in the state words (bits 0), an in-tree bitmap in shared
// memory (1) or in global memory (2), weighted or
// not, popping short cycles from a ring of the last path vertices (ring) or
// walking them, one CTA per tree or a cluster of CTAs per tree (cl; bits 0 or
// 1), for a register cap of 48 or 64 (lower caps map to 48), and its dynamic
// shared memory per CTA in a cluster of C CTAs.
WilsonFn wilson_edge_fn(int bits, bool wgt, bool ring, bool cl, int regs, bool roots = false);
size_t wilson_edge_smem(int W, int32_t n, int bits, bool wgt, int C, bool ring);  // bits: 0 flags, 1 shared bitmap, 2 global

}  // namespace fcx
