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
// One cooperative kernel handles a chunk of up to 32 trees with every
// resident CTA; grid-wide barriers separate the phases, and none of them
// takes a barrier per tree level, so deep trees cost no more barriers than
// shallow ones: child counts (with validation); subtree sizes and sibling
// offsets by peeling leaves (one atomic per tree node, the node finished by
// whichever thread delivers its last child); preorder numbers by pointer
// jumping down the paths (O(log depth) rounds); the rows; and the
// per-vertex sums.  Preorder numbers and sizes are stored vertex-major
// across the chunk's trees, so a warp scanning a row with one lane per tree
// reads each neighbour's numbers for all trees in one 128-byte line.  Long
// unweighted rows are split into segments of 256 entries whose counts add
// up exactly; a weighted row stays with one warp so that each lane adds its
// tree's weights in row order.  Every loop bound and every early exit is
// read from global memory after a barrier, so all CTAs take the same path
// through the barriers.
//
// The same kernel, in its second mode, aggregates the effective resistances
// r(u, v) between a pivot u and every vertex v (Sec. 3, insight (iii)) from
// uniform spanning trees of G rooted at u (sampled on a graph from
// fc_build_rooted, whose trees are u* -> u -> ...).  Kirchhoff's current
// theorem: a unit current from v to u puts current P(a->b) - P(b->a) on an
// edge {a, b}, where P(a->b) is the probability that v's tree path to u
// crosses it from a to b; summing current / w along any fixed path from v to
// u (here v's path in a breadth-first tree B of u) gives r(u, v).  Per tree,
//   S_T(v) = sum over the edges (x, b(x)) of v's B-path, from v upward, of
//            ( [par_T(x) = b(x), x ancestor-or-self of v in T]
//            - [par_T(b(x)) = x, b(x) ancestor-or-self of v in T] ) / w(x, b(x)),
// summed in FP64 in path order and added in signed fixed point
// floor(S_T(v) 2^32 + 1/2).  Ancestry uses the same preorder numbers and
// subtree sizes; a warp takes a vertex and walks its B-path once for the
// chunk's trees (one lane per tree, tree parents stored vertex-major).
#include <cooperative_groups.h>

#include <algorithm>

#include "fc_internal.cuh"

namespace cg = cooperative_groups;

namespace fcx {

namespace {

constexpr int RB_T = 256;
constexpr int RB_FRAC = 48;
constexpr int RB_SEG = 256;  // entries per segment of a long unweighted row
constexpr int RB_TMAX = 32;  // trees per chunk: one per lane of a warp

struct RBParams {
  int32_t n;
  int32_t Tc;                 // trees in this chunk (at most 32: one per lane)
  const int64_t* rowptr;
  const int32_t* colidx;
  const float* w;             // or null
  double alpha;
  const double* alpha_v;      // per-vertex alpha (batches) or null
  const int32_t* parents;     // [Tc][n]
  uint64_t* acc;              // [n] fixed-point sums
  const int4* segs;           // row segments {v, entries, first entry (low, high word)}
  const uint32_t* nseg;       // number of segments
  // scratch.  Per tree node flat index i = t (n + 1) + v, where v = n is the
  // tree's u*; vertex-major index v Tc + t.
  uint32_t* cnt;              // [Tc (n + 1)] children counts (zeroed by the host)
  unsigned long long* word;   // [Tc (n + 1)] {summed sizes of finished children, finished children} (zeroed)
  uint32_t* rsz;              // [Tc (n + 1)] subtree size of each root, 0 elsewhere
  unsigned long long* jw;     // [Tc (n + 1)] pointer-jumping words {ancestor, partial preorder number}
  int32_t* size;              // [n][Tc] subtree sizes (vertex-major)
  int32_t* tin;               // [n][Tc] preorder numbers (vertex-major)
  double* sout;               // [n][Tc] weighted: sum over neighbours outside the subtree
  uint32_t* outc;             // [n][Tc] unweighted: count of neighbours outside the subtree
  uint32_t* rsum;             // [Tc (n + 1)] exclusive scan of the roots' subtree sizes
  uint32_t* bsum;             // [gridDim.x] block totals of the scan
  uint32_t* ctr;              // [2] error, [4..6] active counts of the jumping rounds, [7] chunk grabs (zeroed)
  const uint64_t* qtab;       // unweighted, one alpha: fixed-point value for each count of outside neighbours, or null
  // resistance mode
  int32_t root;               // the pivot u (the only child of u*), -1 in the diag(Omega) mode
  const int32_t* bpar;        // [n] breadth-first parent of each vertex (-1 at the root)
  const double* binv;         // [n] 1 / w(v, bpar(v))
  int64_t* racc;              // [n] signed fixed-point totals of S_T(v)
  int32_t* pvm;               // [n][Tc] tree parents, vertex-major
};

constexpr int RES_FRAC = 32;

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

// Grid-wide exclusive scan out[i] = sum_{j < i} val(j) (mod 2^32) over
// [0, len): each CTA scans a contiguous range, CTA 0 scans the range totals,
// and each CTA adds its carry.  Ends without a trailing barrier.
template <class F>
__device__ void grid_exscan(cg::grid_group& grid, F val, uint32_t* out, int64_t len, uint32_t* bsum,
                            uint32_t* wsum, uint32_t* carry) {
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = std::min<int64_t>(len, (int64_t)blockIdx.x * chunk);
  const int64_t b1 = std::min<int64_t>(len, b0 + chunk);
  if (threadIdx.x == 0) *carry = 0;
  __syncthreads();
  for (int64_t base = b0; base < b1; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const uint32_t x = i < b1 ? val(i) : 0u;
    uint32_t tot = 0;
    const uint32_t ex = block_exscan_u32(x, &tot, wsum);
    if (i < b1) out[i] = *carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) *carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = *carry;
  grid.sync();
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) *carry = 0;
    __syncthreads();
    for (int base = 0; base < (int)gridDim.x; base += blockDim.x) {
      const int j = base + threadIdx.x;
      const uint32_t x = j < (int)gridDim.x ? bsum[j] : 0u;
      uint32_t tot = 0;
      const uint32_t ex = block_exscan_u32(x, &tot, wsum);
      if (j < (int)gridDim.x) bsum[j] = *carry + ex;
      __syncthreads();
      if (threadIdx.x == 0) *carry += tot;
      __syncthreads();
    }
  }
  grid.sync();
  const uint32_t add = bsum[blockIdx.x];
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) out[i] += add;
}

__device__ __forceinline__ unsigned long long jw_pack(int32_t anc, int32_t sum) {
  return (unsigned long long)(uint32_t)anc | ((unsigned long long)(uint32_t)sum << 32);
}

constexpr int RB_TILE = 256;  // vertices per tile of the vertex-major transpose

// MODE 0: Rao-Blackwellised diag(Omega); MODE 1: effective resistances to the pivot.
template <int MODE>
__global__ void __launch_bounds__(RB_T, 5) k_rb(RBParams p) {
  cg::grid_group grid = cg::this_grid();
  __shared__ int32_t tile[RB_TMAX][RB_TILE + 1];
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  const int32_t n = p.n;
  const int32_t n1 = n + 1;
  const int32_t Tc = p.Tc;
  const int64_t N1 = (int64_t)Tc * n1;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = gtid >> 5, nwarps = gstride >> 5;
#define VT(t, v) ((int64_t)(v) * Tc + (t))

  // ---- child counts; parents must lie in [0, n] and differ from the vertex ----
  for (int64_t i = gtid; i < N1; i += gstride) {
    const int32_t t = (int32_t)(i / n1), v = (int32_t)(i - (int64_t)t * n1);
    p.rsz[i] = 0u;
    if (v == n) {
      p.jw[i] = jw_pack(-1, -1);
      continue;
    }
    const int32_t par = p.parents[(int64_t)t * n + v];
    if (par < 0 || par > n || par == v) atomicOr(&p.ctr[2], ERR_INVAL);
    // a tree of G rooted at the pivot: the pivot, and only the pivot, hangs from u*
    else if (MODE == 1 && ((par == n) != (v == p.root))) atomicOr(&p.ctr[2], ERR_INVAL);
    else if (par < n) atomicAdd(&p.cnt[(int64_t)t * n1 + par], 1u);  // u*'s children: a scan below
  }
  grid.sync();
  if (*(volatile uint32_t*)&p.ctr[2] != 0u) return;  // uniform: read after the barrier

  // ---- subtree sizes and sibling offsets by peeling leaves.  A finished
  // child adds {its size, 1} to its parent's word in one atomic; the sizes
  // already there are its earlier-finished siblings', so 1 + that sum is its
  // offset in the parent's preorder interval (any sibling order gives valid
  // intervals, and subtree membership does not depend on it).  The thread
  // that delivers a parent's last child carries on with the parent: no
  // barrier per tree level.  The roots (u*'s children, often most vertices)
  // take their offsets from a scan instead of one contended word. ----
  // Warps take candidates in chunks of 32 (coalesced, one chunk ahead)
  // from a shared counter, eight chunks per grab, and hand the leaves among
  // them to whichever lanes are idle.  The last deliverer of a node carries
  // on with it, so chains pile up on some lanes; warps so held up take fewer
  // chunks, and the rest of their lanes keep taking leaves.  A step loads the
  // parent's child count and the grandparent before its atomic, so all three
  // are in flight together.
  {
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nchunks = (N1 + 31) / 32;
    int64_t sc = 0;  // current grab (warp-uniform)
    int kc = 8;      // next chunk within it
    bool dry = false;
    auto next_chunk = [&]() -> int64_t {
      if (dry) return -1;
      if (kc == 8) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&p.ctr[7], 1u);
        sc = __shfl_sync(0xffffffffu, g, 0);
        kc = 0;
      }
      const int64_t c = sc * 8 + kc++;
      if (c >= nchunks) dry = true;
      return dry ? -1 : c;
    };
    int32_t nt = 0, nv = n, np = 0;  // prefetched chunk: this lane's node
    uint32_t nc = 1u;
    bool pre = false;  // a prefetched chunk is waiting (warp-uniform)
    auto load = [&]() {
      const int64_t c = next_chunk();
      pre = c >= 0;
      nt = 0;
      nv = n;
      nc = 1u;
      np = 0;
      const int64_t i = c * 32 + lane;
      if (pre && i < N1) {
        nt = (int32_t)(i / n1);
        nv = (int32_t)(i - (int64_t)nt * n1);
        if (nv != n) {
          nc = p.cnt[i];
          np = p.parents[(int64_t)nt * n + nv];
        }
      }
    };
    load();
    unsigned lmask = 0;  // leaves of the current chunk not yet taken (warp-uniform)
    int32_t ct = 0, cv = 0, cpar = 0;  // this lane's node of the current chunk
    int32_t t = -1, v = 0, par = 0;
    uint32_t s = 0;
    for (;;) {
      if (lmask == 0u && pre) {  // the prefetched chunk becomes current
        ct = nt;
        cv = nv;
        cpar = np;
        lmask = __ballot_sync(0xffffffffu, nv != n && nc == 0u);
        load();
      }
      const unsigned need = __ballot_sync(0xffffffffu, t < 0);
      if (need == 0xffffffffu && lmask == 0u && !pre) break;  // uniform
      const int avail = __popc(lmask);
      const int ntake = min(__popc(need), avail);
      const int r = __popc(need & lt);
      const bool take = t < 0 && r < avail;
      const int src = take ? (int)__fns(lmask, 0, r + 1) : lane;
      const int32_t tt = __shfl_sync(0xffffffffu, ct, src);
      const int32_t tv = __shfl_sync(0xffffffffu, cv, src);
      const int32_t tp = __shfl_sync(0xffffffffu, cpar, src);
      // the first ntake leaves are taken
      lmask = ntake == avail ? 0u : lmask & ~((1u << __fns(lmask, 0, ntake + 1)) - 1u);
      if (take) {
        t = tt;
        v = tv;
        par = tp;
        s = 1u;
        p.size[VT(t, v)] = 1;
      }
      if (t < 0) continue;
      if (par == n) {  // a root: its offset comes from the scan below
        p.rsz[(int64_t)t * n1 + v] = s;
        t = -1;
        continue;
      }
      const int64_t pi = (int64_t)t * n1 + par;
      const uint32_t cp = p.cnt[pi];
      const int32_t gp = p.parents[(int64_t)t * n + par];
      const unsigned long long old = atomicAdd(&p.word[pi], (1ull << 32) | s);
      p.jw[(int64_t)t * n1 + v] = jw_pack((int32_t)pi, (int32_t)(1u + (uint32_t)old));
      if ((uint32_t)(old >> 32) + 1u != cp) {
        t = -1;
        continue;
      }
      s = 1u + (uint32_t)old + s;
      v = par;
      par = gp;
      p.size[VT(t, v)] = (int32_t)s;
    }
  }
  grid.sync();
  // roots in vertex order: preorder number = sizes of the tree's earlier roots
  grid_exscan(grid, [&](int64_t i) { return p.rsz[i]; }, p.rsum, N1, p.bsum, wsum, &carry);
  grid.sync();
  for (int64_t i = gtid; i < N1; i += gstride) {
    const int32_t t = (int32_t)(i / n1), v = (int32_t)(i - (int64_t)t * n1);
    const uint32_t base = p.rsum[(int64_t)t * n1];
    if (v == n) {
      // a parent cycle leaves its vertices and their subtrees outside u*'s tree
      if (p.rsum[i] - base != (uint32_t)n) atomicOr(&p.ctr[2], ERR_INVAL);
    } else if (p.rsz[i] != 0u) {
      p.jw[i] = jw_pack(-1, (int32_t)(p.rsum[i] - base));
    }
  }
  grid.sync();
  if (*(volatile uint32_t*)&p.ctr[2] != 0u) return;

  // ---- preorder numbers: each node's number is its parent's plus its
  // offset, summed down the path by pointer jumping.  Invariant: tin(i) =
  // sum(i) + tin(anc(i)), with anc = -1 once sum is the number itself; words
  // are read and written whole, so a node may read an ancestor's word of
  // this round or the last one.  O(log depth) rounds. ----
  for (int r = 0;; ++r) {
    uint32_t active = 0;
    for (int64_t i = gtid; i < N1; i += gstride) {
      volatile unsigned long long* jv = p.jw;
      const unsigned long long w0 = jv[i];
      const int32_t a = (int32_t)(uint32_t)w0;
      if (a < 0) continue;
      const unsigned long long w1 = jv[a];
      const int32_t a1 = (int32_t)(uint32_t)w1;
      jv[i] = jw_pack(a1, (int32_t)((uint32_t)(w0 >> 32) + (uint32_t)(w1 >> 32)));
      active += a1 >= 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) active += __shfl_xor_sync(0xffffffffu, active, o);
    if (lane == 0 && active) atomicAdd(&p.ctr[4 + r % 3], active);
    if (gtid == 0) p.ctr[4 + (r + 1) % 3] = 0u;  // read two rounds ago, after that round's barrier
    grid.sync();
    if (*(volatile uint32_t*)&p.ctr[4 + r % 3] == 0u) break;  // uniform
    if (r >= 64) {  // depth below 2^31 needs at most 32 rounds
      if (gtid == 0) atomicOr(&p.ctr[2], ERR_INVAL);
      return;
    }
  }
  // preorder numbers to vertex-major order through a shared-memory tile
  // (coalesced on both sides); the per-row sums start at zero
  for (int64_t v0 = (int64_t)blockIdx.x * RB_TILE; v0 < n; v0 += (int64_t)gridDim.x * RB_TILE) {
    const int32_t nv = (int32_t)std::min<int64_t>(RB_TILE, n - v0);
    for (int t = 0; t < Tc; ++t)
      for (int x = threadIdx.x; x < nv; x += blockDim.x) tile[t][x] = (int32_t)(p.jw[(int64_t)t * n1 + v0 + x] >> 32);
    __syncthreads();
    const int64_t k1 = (int64_t)nv * Tc;
    for (int64_t k = threadIdx.x; k < k1; k += blockDim.x) {
      const int32_t x = (int32_t)(k / Tc), t = (int32_t)(k - (int64_t)x * Tc);
      p.tin[v0 * Tc + k] = tile[t][x];
      if (MODE == 0) {
        if (p.w) p.sout[v0 * Tc + k] = 0.0;
        else p.outc[v0 * Tc + k] = 0u;
      }
    }
    __syncthreads();
    if (MODE == 1) {  // the tree parents, vertex-major, through the same tile
      for (int t = 0; t < Tc; ++t)
        for (int x = threadIdx.x; x < nv; x += blockDim.x) tile[t][x] = p.parents[(int64_t)t * n + v0 + x];
      __syncthreads();
      for (int64_t k = threadIdx.x; k < k1; k += blockDim.x) {
        const int32_t x = (int32_t)(k / Tc), t = (int32_t)(k - (int64_t)x * Tc);
        p.pvm[v0 * Tc + k] = tile[t][x];
      }
      __syncthreads();
    }
  }
  grid.sync();

  if (MODE == 1) {
    // ---- path sums along the breadth-first tree: a warp per vertex, a lane
    // per tree; the B-path is the same for every lane ----
    const int32_t root = p.root;
    for (int64_t v = gwarp; v < n; v += nwarps) {
      const bool on = lane < Tc;
      const int32_t tv = on ? p.tin[VT(lane, v)] : 0;
      double s = 0.0;
      int32_t x = (int32_t)v;
      int32_t px = on ? p.pvm[VT(lane, x)] : -1;  // parent of x in this lane's tree
      int32_t hops = 0;
      while (x != root) {
        const int32_t b = __ldg(p.bpar + x);
        const double wi = __ldg(p.binv + x);
        if (b < 0 || ++hops > n) {  // not a breadth-first tree of the root: never for fc_build_rooted graphs
          atomicOr(&p.ctr[2], ERR_INVAL);
          break;
        }
        const int32_t pb = (on && b != root) ? p.pvm[VT(lane, b)] : -1;  // parent of b
        if (on) {
          int c = 0;
          if (px == b) {  // the tree crosses x -> b: on v's tree path iff x is an ancestor-or-self of v
            const int32_t t0 = p.tin[VT(lane, x)];
            if (t0 <= tv && tv < t0 + p.size[VT(lane, x)]) c = 1;
          } else if (pb == x) {  // the tree crosses b -> x
            const int32_t t0 = p.tin[VT(lane, b)];
            if (t0 <= tv && tv < t0 + p.size[VT(lane, b)]) c = -1;
          }
          if (c != 0) s = __dadd_rn(s, c > 0 ? wi : -wi);
        }
        x = b;
        px = pb;
      }
      long long q = 0;
      if (on) q = (long long)floor(__dadd_rn(__dmul_rn(s, (double)(1ull << RES_FRAC)), 0.5));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if (lane == 0 && q != 0) atomicAdd((unsigned long long*)&p.racc[v], (unsigned long long)q);
    }
    return;
  }

  // ---- neighbours outside the subtree: a warp per row segment, a lane per
  // tree (each lane sums its tree's weights in row order; unweighted counts
  // of the segments of a long row add up exactly) ----
  // The next segment's record is loaded while the current one is scanned.
  const int64_t nseg = *p.nseg;
  int4 nxt = gwarp < nseg ? p.segs[gwarp] : make_int4(0, 0, 0, 0);
  for (int64_t sg = gwarp; sg < nseg; sg += nwarps) {
    const int4 sv = nxt;
    if (sg + nwarps < nseg) nxt = p.segs[sg + nwarps];
    const int32_t v = sv.x;
    const int64_t e0 = (int64_t)(((uint64_t)(uint32_t)sv.w << 32) | (uint32_t)sv.z);
    const int64_t e1 = e0 + sv.y;
    const bool on = lane < Tc;
    int32_t lo = 0, hi = 0;
    if (on) {
      lo = p.tin[VT(lane, v)];
      hi = lo + p.size[VT(lane, v)];
    }
    double s = 0.0;
    uint32_t c = 0;
    // 32 entries at a time: lane j loads entry j, the warp broadcasts them
    // and each lane tests its own tree, in row order; the preorder numbers of
    // eight neighbours are loaded before any is tested, so eight loads are in
    // flight (a neighbour past the row's end reads as inside the subtree)
    for (int64_t eb = e0; eb < e1; eb += 32) {
      const int32_t m = (int32_t)std::min<int64_t>(32, e1 - eb);
      const int32_t uj = lane < m ? __ldg(p.colidx + eb + lane) : 0;
      const float wj = (p.w && lane < m) ? __ldg(p.w + eb + lane) : 0.f;
      for (int k0 = 0; k0 < m; k0 += 8) {
        int32_t tu[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int32_t u = __shfl_sync(0xffffffffu, uj, (k0 + kk) & 31);
          tu[kk] = (on && k0 + kk < m) ? p.tin[VT(lane, u)] : lo;
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float wk = __shfl_sync(0xffffffffu, wj, (k0 + kk) & 31);
          if (tu[kk] < lo || tu[kk] >= hi) {
            if (p.w) s = __dadd_rn(s, (double)wk);
            else ++c;
          }
        }
      }
    }
    if (on) {
      if (p.w) p.sout[VT(lane, v)] = s;  // weighted rows are one segment
      else if (c) atomicAdd(&p.outc[VT(lane, v)], c);
    }
  }
  grid.sync();

  // ---- the conditional probabilities, summed over the chunk's trees ----
  for (int64_t v = gwarp; v < n; v += nwarps) {
    uint64_t q = 0;
    if (lane < Tc && p.qtab) {
      q = p.qtab[p.outc[VT(lane, v)]];  // the same FP64 steps, done once per count
    } else if (lane < Tc) {
      const double s = p.w ? p.sout[VT(lane, v)] : (double)p.outc[VT(lane, v)];
      const double a = p.alpha_v ? p.alpha_v[v] : p.alpha;
      const double val = __ddiv_rn(1.0, __dadd_rn(1.0, __dmul_rn(a, s)));
      q = (uint64_t)__dadd_rn(__dmul_rn(val, (double)(1ull << RB_FRAC)), 0.5);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) atomicAdd((unsigned long long*)&p.acc[v], (unsigned long long)q);
  }
#undef VT
}

// Fixed-point value of 1 / (1 + alpha c) for every count c = 0..cmax of
// outside neighbours (unweighted graphs, one alpha), with the FP64 steps of
// the per-tree formula, so a table lookup gives the same bits.
__global__ void k_rb_table(double alpha, int32_t cmax, uint64_t* __restrict__ qtab) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= cmax; c += (int64_t)gridDim.x * blockDim.x) {
    const double val = __ddiv_rn(1.0, __dadd_rn(1.0, __dmul_rn(alpha, (double)c)));
    qtab[c] = (uint64_t)__dadd_rn(__dmul_rn(val, (double)(1ull << RB_FRAC)), 0.5);
  }
}

__global__ void k_rb_diag(int32_t n, const uint64_t* __restrict__ acc, double denom, double* __restrict__ diag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    diag[v] = __ddiv_rn((double)acc[v], denom);
}

// Segments per row: unweighted rows split every RB_SEG entries (their
// integer counts add up exactly); weighted rows stay whole so that each
// tree's sum keeps the row order.  cnt has n + 1 entries, the last 0.
__global__ void k_seg_count(int32_t n, const int64_t* __restrict__ rowptr, bool weighted, uint32_t* __restrict__ cnt) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c = 0;
    if (v < n) {
      const int64_t d = rowptr[v + 1] - rowptr[v];
      c = weighted ? (d > 0 ? 1u : 0u) : (uint32_t)((d + RB_SEG - 1) / RB_SEG);
    }
    cnt[v] = c;
  }
}

__global__ void k_seg_fill(int32_t n, const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off,
                           const int64_t* __restrict__ rowptr, bool weighted, int4* __restrict__ segs) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t o = off[v];
    const int64_t r0 = rowptr[v], r1 = rowptr[v + 1];
    for (uint32_t k = 0; k < cnt[v]; ++k) {
      const int64_t e0 = r0 + (int64_t)k * RB_SEG;
      const int32_t m = (int32_t)(weighted ? r1 - r0 : std::min<int64_t>(RB_SEG, r1 - e0));
      segs[o + k] = make_int4((int32_t)v, m, (int32_t)(uint32_t)e0, (int32_t)(uint32_t)((uint64_t)e0 >> 32));
    }
  }
}

}  // namespace

}  // namespace fcx

using namespace fcx;

// Chunks of up to 32 trees through k_rb<mode>: mode 0 adds the
// Rao-Blackwellised values to acc (uint64), mode 1 the path sums S_T(v) to
// acc (int64).
static fc_status tree_chunks(fc_graph* g, int mode, int32_t alpha_idx, const int32_t* parents, int64_t T, void* acc,
                             cudaStream_t st, const char* who) {
  const int32_t n = g->n;
  int dev = g->device, nsm = 0, coop = 0, per_sm = 0;
  FC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FC_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) {
    set_error(std::string(who) + ": the device does not support cooperative launches");
    return FC_ECUDA;
  }
  const void* kern = mode == 0 ? (const void*)k_rb<0> : (const void*)k_rb<1>;
  FC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RB_T, 0));
  const int grid = std::max(1, per_sm) * nsm;  // every CTA resident: required by the grid barriers
  // trees per chunk: one per lane, 44 bytes of scratch per (tree, vertex)
  // within a sixteenth of the device (1 to 16 GB), flat ids below 2^31
  const int64_t budget = std::max<int64_t>(1ll << 30, std::min<int64_t>(16ll << 30, (int64_t)(g->device_bytes / 16)));
  const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(budget / (44ll * (n + 1)),
                                                             ((int64_t)1 << 31) / ((int64_t)n + 1) - 1));
  const int64_t Tc_max = std::min<int64_t>(std::min<int64_t>(T, RB_TMAX), cap);
  const size_t N1 = (size_t)Tc_max * (n + 1), N = (size_t)Tc_max * n;
  const int64_t seg_max = (int64_t)n + g->nnz / RB_SEG + 1;  // bound on the number of segments
  char* ws = nullptr;
  const size_t bytes = N1 * 4 * 3 + (size_t)grid * 4 + N1 * 8 * 2 + N * 4 * 2 + N * 8 + 32 +
                       ((size_t)n + 1) * 8 + (size_t)seg_max * 16 + ((size_t)g->max_deg + 1) * 8 + 256 * 16;
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
  p.acc = mode == 0 ? (uint64_t*)acc : nullptr;
  p.racc = mode == 1 ? (int64_t*)acc : nullptr;
  p.root = mode == 1 ? g->root : -1;
  p.bpar = g->bpar;
  p.binv = g->binv;
  p.cnt = (uint32_t*)carve(N1 * 4);
  p.word = (unsigned long long*)carve(N1 * 8);
  p.rsz = (uint32_t*)carve(N1 * 4);
  p.jw = (unsigned long long*)carve(N1 * 8);
  p.size = (int32_t*)carve(N * 4);
  p.tin = (int32_t*)carve(N * 4);
  p.sout = (double*)carve(N * 8);  // the unweighted counts use its first half
  p.outc = (uint32_t*)p.sout;
  p.pvm = (int32_t*)p.sout;        // resistance mode: the tree parents, vertex-major
  p.rsum = (uint32_t*)carve(N1 * 4);
  p.bsum = (uint32_t*)carve((size_t)grid * 4);
  p.ctr = (uint32_t*)carve(32);
  const bool table = mode == 0 && g->w == nullptr && g->num_graphs == 0;
  uint64_t* qtab = table ? (uint64_t*)carve(((size_t)g->max_deg + 1) * 8) : nullptr;
  p.qtab = qtab;
  uint32_t* scnt = (uint32_t*)carve(((size_t)n + 1) * 4);
  uint32_t* soff = (uint32_t*)carve(((size_t)n + 1) * 4);
  int4* segs = (int4*)carve((size_t)seg_max * 16);
  ws = base;
  p.segs = segs;
  p.nseg = soff + n;
  if (mode == 0) {  // row segments (the resistance mode reads no rows)
    const unsigned b = (unsigned)std::min<int64_t>(((int64_t)n + 256) / 256, (int64_t)nsm * 16);
    k_seg_count<<<b, 256, 0, st>>>(n, g->rowptr, g->w != nullptr, scnt);
    FC_LAUNCHED();
    const fc_status r = exclusive_scan(scnt, soff, (int64_t)n + 1, st);
    if (r != FC_OK) {
      FC_CK(cudaFreeAsync(base, st));
      return r;
    }
    k_seg_fill<<<b, 256, 0, st>>>(n, scnt, soff, g->rowptr, g->w != nullptr, segs);
    FC_LAUNCHED();
    if (table) {
      const unsigned bt = (unsigned)std::min<int64_t>(((int64_t)g->max_deg + 256) / 256, (int64_t)nsm * 4);
      k_rb_table<<<bt, 256, 0, st>>>(p.alpha, g->max_deg, qtab);
      FC_LAUNCHED();
    }
  }
  fc_status status = FC_OK;
  for (int64_t t0 = 0; t0 < T && status == FC_OK; t0 += Tc_max) {
    const int32_t Tc = (int32_t)std::min<int64_t>(Tc_max, T - t0);
    p.Tc = Tc;
    p.parents = parents + (size_t)t0 * n;
    FC_CK(cudaMemsetAsync(p.cnt, 0, (size_t)Tc * (n + 1) * 4, st));
    FC_CK(cudaMemsetAsync(p.word, 0, (size_t)Tc * (n + 1) * 8, st));
    FC_CK(cudaMemsetAsync(p.ctr, 0, 32, st));
    void* args[] = {&p};
    FC_CK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(RB_T), args, 0, st));
    FC_LAUNCHED();
    uint32_t herr = 0;
    FC_CK(cudaMemcpyAsync(&herr, p.ctr + 2, 4, cudaMemcpyDeviceToHost, st));
    FC_CK(cudaStreamSynchronize(st));
    if (herr != 0) {
      set_error(std::string(who) + (mode == 0 ? ": parents do not form spanning trees of G* rooted at u* = n"
                                              : ": parents do not form spanning trees of G rooted at the pivot"));
      status = FC_EINVAL;
    }
  }
  FC_CK(cudaFreeAsync(base, st));
  return status;
}

extern "C" fc_status fc_rb_accumulate(fc_graph* g, int32_t alpha_idx, const int32_t* parents, int64_t T,
                                      uint64_t* acc, void* stream) {
  if (g == nullptr || parents == nullptr || acc == nullptr || T < 0 || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha) {
    set_error("fc_rb_accumulate: bad argument");
    return FC_EINVAL;
  }
  if (T == 0) return FC_OK;
  return tree_chunks(g, 0, alpha_idx, parents, T, acc, (cudaStream_t)stream, "fc_rb_accumulate");
}

extern "C" fc_status fc_resistance_accumulate(fc_graph* g, const int32_t* parents, int64_t T, int64_t* acc,
                                              void* stream) {
  if (g == nullptr || parents == nullptr || acc == nullptr || T < 0) {
    set_error("fc_resistance_accumulate: bad argument");
    return FC_EINVAL;
  }
  if (g->root < 0 || g->bpar == nullptr) {
    set_error("fc_resistance_accumulate: needs a graph from fc_build_rooted");
    return FC_EINVAL;
  }
  if (T == 0) return FC_OK;
  return tree_chunks(g, 1, 0, parents, T, acc, (cudaStream_t)stream, "fc_resistance_accumulate");
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
