// Edge-record variant of the Wilson sampler (Algorithm 2 on G*, rooted at u*)
// for single graphs with the per-tree state in global memory.
//
// It uses the same random stacks, the same cycle-popping argument (so the
// trees are bit-identical to the sequential sampler's) and the same wait-die
// protocol as the CSR-walk kernel; what differs is the memory schedule of a
// walk step, which decides the speed of this latency-bound loop.
//
//  * Each CSR entry is widened to a 16-byte record describing its target:
//    {vertex, row offset, degree, high 32 bits of its u*-threshold T}.  A
//    walker that steps onto x therefore already holds x's row: it computes
//    x's stack entry for k = 0 speculatively and loads the selected record in
//    the same round trip as the CAS that claims x.
//  * Tree membership is a flag bit in x's state word, set when a path joins
//    the tree, so that same CAS also answers "is x in the tree?".  One
//    dependent round trip per step instead of two, and no per-tree bitmap.
//  * The slot decision stays exact: with T_hi = min(T >> 21, 2^32 - 1) and
//    u_hi = u53 >> 21, u_hi < T_hi implies u53 < T and u_hi > T_hi implies
//    u53 >= T; only u_hi == T_hi (probability about 2^-32 per step) reads the
//    full T from the row info.
//  * Start vertices are handed out per warp from windows of 32 consecutive
//    positions of the start order; the warp fetches the 32 row infos (and
//    state words) together (coalesced in vertex-id order) and keeps only the
//    vertices not yet in the tree, compacted to the front of the window.
//
// State word: bits 0..23 k (stack entries popped), bits 24..62 tag
// ((gen << 10) | walker, 0 = free), bit 63 in-tree flag.
#include <cooperative_groups.h>

#include "fc_wilson_common.cuh"

namespace cg = cooperative_groups;

namespace fcx {

namespace {

constexpr unsigned long long IN_TREE = 1ull << 63;
constexpr unsigned long long TAG_MASK = (1ull << (63 - K_BITS)) - 1ull;

enum { E_IDLE = 0, E_START, E_THR, E_CLAIM, E_CLAIM2, E_TOP, E_POP, E_RETRACE, E_RELEASE, E_WAIT, E_DONE };

// Walker ids are tree-wide (a tree may span a cluster of up to 8 CTAs of up
// to 1024 walkers); the tag's generation gets the remaining 26 bits.
constexpr int EW_BITS = 13;
constexpr uint32_t EW_MASK = (1u << EW_BITS) - 1u;
constexpr uint32_t GEN_LIMIT = (1u << (39 - EW_BITS)) - 1u;
// parked restarts (RINGP): no parked path / parked, a window start to be taken first
constexpr uint32_t NO_PARK = 0xffffffffu;
constexpr uint32_t PARK_FRESH = 0x80000000u;

__device__ __forceinline__ unsigned long long rd_pack(int32_t root, int32_t depth) {
  return (unsigned long long)(uint32_t)root | ((unsigned long long)(uint32_t)depth << 32);
}

__device__ __forceinline__ uint32_t thr_hi(const uint4& ri) {
  const uint64_t T = (uint64_t)ri.z | ((uint64_t)ri.w << 32);
  return T >= (1ull << 53) ? 0xffffffffu : (uint32_t)(T >> 21);
}

// Asynchronous 16-byte global -> shared copies (through L2), used to fetch the
// next start window in the same round trip as the walk step.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace

// BITS: where tree membership lives.  0: the flag bit of the state words (the
// claiming CAS answers "in the tree?").  1: an in-tree bitmap in shared memory
// (graphs whose n/8 bytes fit next to the walker arrays).  2: an in-tree
// bitmap per CTA in global memory (L2-resident for the trees in flight).  With
// a bitmap a claim first tests x's bit and touches neither x's state nor an
// edge record when x is already in the tree, and finished paths are marked in
// the bitmap instead of the state words.
//
// WGT: weighted graphs.  Records are 64 bytes: the 16-byte header above plus
// the high words (bits 32..52) of the target's first 12 slot thresholds B.
// A walker keeps the thresholds of its current vertex in shared memory (two
// buffers: the record of the next vertex is copied into the other one while
// the current vertex is claimed).  A slot is decided from the high words when
// they differ from u53 >> 32 and from the exact B (global memory) on the rare
// tie; rows with more than 13 slots search the rest of B in global memory.
//
// RINGP: the walker's shared-memory path buffer holds its last PB path
// vertices (a ring) instead of the first PB, so a cycle closing within them is
// popped at once without loads (graphs whose walks loop often); otherwise the
// buffer holds the path prefix and every cycle is walked through nxt.
//
// CL: a tree is shared by the C CTAs of a thread-block cluster (launched with
// cluster dimension C; grids of few trees then still fill the GPU, and the
// in-tree bitmap of a large graph fits when split over C shared memories).
// Rank 0 holds the tree index, the start-window counter and the tree's pop
// and departure totals; the bitmap is interleaved by 32-bit word over the
// ranks; walker generations are read across the cluster (distributed shared
// memory).  Cluster barriers separate the trees.
//
// ROOTS: forest roots and depths of every tree (the roots are the children of
// u*), written as vertices join the tree: a path that exits to u* at its head
// h roots all its vertices at h, one that reaches tree vertex x inherits x's
// root, and depths count down the path to the root.  A vertex's root and
// depth are stored before its membership becomes visible (a fence between;
// every reader is a walker of the same CTA, so a CTA-scope fence), so a walker
// that sees x in the tree reads x's final values.
template <int BITS, bool WGT, bool RINGP, bool CL, int MAXREG, bool ROOTS>
__global__ void __launch_bounds__(1024) __maxnreg__(MAXREG) k_wilson_edge(WParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long sh_tree, sh_pops, sh_deps;
  __shared__ uint32_t sh_next, sh_tsize;
  __shared__ volatile uint32_t sh_abort;
  const int me = threadIdx.x;
  const int W = blockDim.x;
  const int lane = me & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  volatile uint32_t* sh_gen = (volatile uint32_t*)smem_raw;               // [W]
  uint32_t* sh_pb = (uint32_t*)(smem_raw + (size_t)W * 4);                // [PB][W] ring of the last path vertices
  // start window of this warp: row info and state record of each slot (copied
  // asynchronously) and its vertex
  uint4* sh_wri = (uint4*)(smem_raw + (((size_t)W * 4 * (1 + PB) + 15) & ~(size_t)15));
  uint4* sh_wst = sh_wri + W;  // BITS = 0 only
  uint32_t* sh_wv = (uint32_t*)(sh_wri + (BITS == 0 ? 2 : 1) * W);
  // RINGP: a path given up under wait-die, parked while its walker takes other
  // start vertices: [W] owner tag of the vertex it met, [W] its start vertex
  // (NO_PARK: none), [W] the vertex it met (sh_wv + W is 16-byte aligned: W is
  // a multiple of 32)
  unsigned long long* sh_ptag = (unsigned long long*)(sh_wv + W);
  uint32_t* sh_ps = (uint32_t*)(sh_ptag + W);
  uint32_t* sh_px = sh_ps + W;
  // [2][W][12] slot-threshold high words of each walker's current / next vertex (WGT)
  uint32_t* sh_thr = (uint32_t*)(((uintptr_t)(RINGP ? (void*)(sh_px + W) : (void*)(sh_wv + W)) + 15) & ~(uintptr_t)15);
  // in-tree bitmap [ceil(n / 32)] (BITS = 1: shared memory, 2: this CTA's global region)
  volatile uint32_t* sh_bits = BITS == 1 ? (volatile uint32_t*)(sh_thr + (WGT ? 2 * 12 * W : 0))
                                         : (volatile uint32_t*)(p.gbits + (size_t)blockIdx.x * p.words);
  // cluster geometry (C = 1 without clusters)
  uint32_t rank = 0, C = 1, clog = 0;
  if (CL) {
    rank = cg::this_cluster().block_rank();
    C = cg::this_cluster().num_blocks();
    clog = (uint32_t)(__ffs((int)C) - 1);  // C is a power of two
  }
  const uint32_t wid = rank * (uint32_t)W + (uint32_t)me;  // walker id within the tree
  const uint32_t WT = C * (uint32_t)W;                     // walkers per tree
  const size_t tslot = CL ? blockIdx.x / C : blockIdx.x;   // tree slot of this CTA
  if (BITS == 2) sh_bits = (volatile uint32_t*)(p.gbits + tslot * p.words);
  uint32_t* my_thr0 = sh_thr + (size_t)me * 12;
  uint32_t* my_thr1 = sh_thr + (size_t)(W + me) * 12;
  sh_wri += me & ~31;
  sh_wst += me & ~31;
  sh_wv += me & ~31;
  const int32_t n = p.n;  // u* = n
  if (p.t0_ns != nullptr && threadIdx.x == 0) atomicMin(p.t0_ns, global_ns());
  VState* S = p.gstate + tslot * p.nmax;
  const int64_t total = (int64_t)(p.num_graphs > 0 ? p.num_graphs : p.n_alpha) * p.tau;  // work items
  bool first_tree = true;

  // Plain memory operations: L2 eviction hints measured slower for this kernel
  // (its 16-byte edge records do not fit in L2 at the sizes where it matters).
#define RING(pos) sh_pb[((pos) & (PB - 1)) * W + me]
  // shared-memory word of another CTA of the cluster (the own one without clusters)
#define REMOTE(ptr, r) (CL ? (volatile uint32_t*)cg::this_cluster().map_shared_rank((uint32_t*)(ptr), (r)) \
                           : (volatile uint32_t*)(ptr))
  // the in-tree bitmap word of vertex v
#define BITW(v) ((BITS == 1 && CL) ? REMOTE(&sh_bits[((uint32_t)((v) - base) >> 5) >> clog],          \
                                          ((uint32_t)((v) - base) >> 5) & (C - 1))                   \
                                   : &sh_bits[(uint32_t)((v) - base) >> 5])
  // the step just taken lands on a vertex already in the tree (bitmap modes):
  // the path is finished in this iteration instead of at the next claim (the
  // bitmap only gains bits, so the answer is final)
#define EARLY_HIT(v) (BITS != 0 && ((*BITW(v) >> ((v) & 31)) & 1u))
  // current generation of walker w of this tree
#define GEN_OF(w) (CL ? *REMOTE(&sh_gen[(w) % (uint32_t)W], (w) / (uint32_t)W) : sh_gen[(w)])
  // stop every CTA working on this tree
#define ABORT_TREE()                                                     \
  do {                                                                   \
    if (CL) {                                                            \
      for (uint32_t r_ = 0; r_ < C; ++r_) *REMOTE(&sh_abort, r_) = 1u;   \
    } else {                                                             \
      sh_abort = 1u;                                                     \
    }                                                                    \
  } while (0)
  // state record of vertex v (global id) in this tree's slot; a batch tree
  // covers the vertex range [base, base + nl) of its graph
#define SV(v) S[(v) - base]
#define ADD_ST(v, d) atomicAdd(&SV(v).st, (d))
#define OR_ST(v, f) atomicOr(&SV(v).st, (f))
#define LD_NXT(v) SV(v).nxt
#define ST_NXT(v, t) (SV(v).nxt = (t))

  for (;;) {
    unsigned long long tree;
    if (!CL) {
      if (me == 0) sh_tree = atomicAdd(p.counter, 1ull);
      __syncthreads();
      tree = sh_tree;
      if ((int64_t)tree >= total || *(volatile uint32_t*)p.err != 0u) break;
    } else {
      // rank 0 takes the next tree (or ends the loop for the whole cluster)
      if (rank == 0 && me == 0) {
        const unsigned long long t = atomicAdd(p.counter, 1ull);
        sh_tree = *(volatile uint32_t*)p.err != 0u ? (unsigned long long)total : t;
      }
      cg::this_cluster().sync();
      tree = *(volatile unsigned long long*)cg::this_cluster().map_shared_rank(&sh_tree, 0u);
      cg::this_cluster().sync();  // every CTA has read rank 0's value
      if ((int64_t)tree >= total) break;
    }
    // item -> (alpha index or graph, tree); the tree's vertices are [base, base + nl)
    int a = (int)(tree / (unsigned long long)p.tau);
    const int64_t tloc = (int64_t)(tree % (unsigned long long)p.tau);
    const uint32_t tg = (uint32_t)(p.tree_offset + tloc);
    int32_t base = 0, nl = n, gi = 0;
    if (p.num_graphs > 0) {
      gi = p.gorder[a];
      a = 0;
      base = (int32_t)p.voff[gi];
      nl = (int32_t)(p.voff[gi + 1] - p.voff[gi]);
    }
    if (!(first_tree && p.pre_cleared))
      for (int32_t v = (int32_t)wid; v < nl; v += (int32_t)WT)
        reinterpret_cast<uint4&>(S[v]) = make_uint4(0u, 0u, 0u, 0u);
    if (BITS == 1)  // this CTA's share of the words (all of them without clusters)
      for (int32_t q = me; q < ((((nl + 31) >> 5) + (int32_t)C - 1) >> clog); q += W) sh_bits[q] = 0u;
    if (BITS == 2 && !(first_tree && p.pre_cleared))
      for (int32_t q = (int32_t)wid; q < ((nl + 31) >> 5); q += (int32_t)WT) sh_bits[q] = 0u;
    first_tree = false;
    sh_gen[me] = 1u;
    if (RINGP) sh_ps[me] = NO_PARK;
    if (me == 0) {
      sh_next = 0;
      sh_tsize = 0;
      sh_abort = 0;
      sh_pops = 0;
      sh_deps = 0;
    }
    if (CL) cg::this_cluster().sync();
    else __syncthreads();
    const uint4* __restrict__ rinfo = p.rowinfo + (size_t)a * n;
    // {root, depth} of this tree's vertices, packed (root low word), by local index
    unsigned long long* RD = ROOTS ? p.rdpack + tslot * (size_t)p.nmax : nullptr;
    const uint4* __restrict__ edges = p.edges + (size_t)a * p.nnz * (WGT ? 4 : 1);
    const uint64_t* __restrict__ Brow = WGT ? p.B + (size_t)a * p.nnz : nullptr;

    int mode = E_IDLE;
    int32_t x = 0, h = -1, c = 0, rh = 0, s = 0, len = 0;
    int32_t rbase = 0;  // path positions [rbase, len) are in the ring (len - rbase <= PB)
    uint32_t xo = 0, xd = 0, xth = 0;  // row offset, degree and T_hi of x
    uint32_t cur = 0;                  // WGT: buffer holding x's slot thresholds
    bool rskip = false;
    bool fexit = false;                             // ROOTS: the finished path left to u*
    int32_t froot = 0, fdl = 0, flen = 0, fpos = 0;  // ROOTS: root, depth base, length, position
    uint32_t gen = 1, kx = 0, iters = 0, pops = 0, deps = 0;
    unsigned long long wtag = 0, cexp = 0;
    uint32_t whead = 0, wcnt = 0;  // warp-uniform: window entries [whead, wcnt) not handed out yet
    bool wdone = false;   // warp-uniform: the start order is exhausted
#if FC_WILSON_COUNTERS
    uint32_t cnt[N_CNT];
#pragma unroll
    for (int q = 0; q < N_CNT; ++q) cnt[q] = 0;
#endif

    while (true) {
      __syncwarp();
      const bool fin = (mode == E_DONE) || (sh_abort != 0u);
      if (__all_sync(FULL, fin)) break;
      // walker ramp (walks on G with one exit): while the tree is small,
      // concurrent walks are long and cross each other, and wait-die makes
      // them repeat work; a warp whose walkers are all idle waits until the
      // tree has grown (or every start position is handed out)
      if (!CL && p.ramp_q != 0u) {
        // lane 0's reading of the shared counters decides for the whole warp
        bool gated = (uint32_t)(me >> 5) > *(volatile uint32_t*)&sh_tsize / p.ramp_q &&
                     *(volatile uint32_t*)&sh_next < (uint32_t)nl;
        gated = __shfl_sync(FULL, gated, 0);
        if (__all_sync(FULL, gated && mode == E_IDLE)) {
          __nanosleep(256);
          continue;
        }
      }

      // ---- start vertices: hand out the window; a dry window is refilled by
      // copies issued with this iteration's memory operations ----
      bool need = !fin && mode == E_IDLE;
      // RINGP: a parked path is looked at again (E_WAIT: has the walker it met
      // moved on?) once its walker has taken one other start vertex, or when no
      // other start vertex is left
      uint32_t pv = NO_PARK;
      if (RINGP && need) {
        pv = sh_ps[me];
        if (pv != NO_PARK && !(pv & PARK_FRESH)) {
          s = (int32_t)pv;
          x = (int32_t)sh_px[me];
          wtag = sh_ptag[me];
          mode = E_WAIT;
          need = false;
        } else if (pv != NO_PARK) {
          sh_ps[me] = pv & ~PARK_FRESH;  // a window start first
        }
      }
      const unsigned want = __ballot_sync(FULL, need);
      bool refill = false;  // warp-uniform
      if (want) {
        const uint32_t nw = (uint32_t)__popc(want), na = wcnt - whead;
        if (need) {
          const uint32_t r = (uint32_t)__popc(want & lt_mask);
          if (r < na) {
            const uint32_t slot = whead + r;
            const uint4 wr = sh_wri[slot];
            s = x = (int32_t)sh_wv[slot];
            xo = wr.x;
            xd = wr.y;
            xth = thr_hi(wr);
            h = -1;
            len = 0;
            rbase = 0;
            mode = WGT ? E_THR : E_CLAIM;
          } else if (wdone) {
            if (RINGP && pv != NO_PARK) {  // nothing else left: wait for the parked path
              s = (int32_t)(pv & ~PARK_FRESH);
              x = (int32_t)sh_px[me];
              wtag = sh_ptag[me];
              mode = E_WAIT;
            } else {
              mode = E_DONE;
            }
          }
        }
        whead = nw >= na ? wcnt : whead + nw;
        refill = nw > na && !wdone;
      }
      bool act = !fin && mode != E_IDLE && mode != E_DONE;
      if (act) {
        CNT(CNT_ITER);
        if (++iters > p.max_iters) {
          atomicOr(p.err, ERR_TIMEOUT);
          ABORT_TREE();
          mode = E_DONE;
          act = false;
        }
      } else {
        CNT(CNT_IDLE_LANE);
      }
      uint32_t wb = 0;
      bool wok = false;
      if (refill) {
        __syncwarp();  // the slots handed out above are read before they are overwritten
        if (lane == 0) wb = atomicAdd(CL ? cg::this_cluster().map_shared_rank(&sh_next, 0u) : &sh_next, 32u);
        wb = __shfl_sync(FULL, wb, 0);
        const uint32_t i = wb + (uint32_t)lane;
        wok = i < (uint32_t)nl;
        if (wok) {
          const uint32_t ix = p.descending ? (uint32_t)nl - 1u - i : i;
          int32_t v = p.id_order ? base + (int32_t)ix : __ldg(p.order + base + ix);
          if (v < base || v >= base + nl) {  // the start order must stay inside the tree's vertex range
            atomicOr(p.err, ERR_INVAL);
            ABORT_TREE();
            v = base;
          }
          sh_wv[lane] = (uint32_t)v;
          cp_async16(&sh_wri[lane], rinfo + v);
          if (BITS == 0) cp_async16(&sh_wst[lane], &SV(v));
        }
        cp_async_commit();
      }

      if (act) {
        const unsigned long long mytag = ((unsigned long long)gen << EW_BITS) | wid;
        uint32_t* thr_cur = cur ? my_thr1 : my_thr0;
        uint32_t* thr_nxt = cur ? my_thr0 : my_thr1;
        if (WGT) cp_async_wait_all();  // x's thresholds, copied during the previous step

        // ---- issue: claim x and, speculatively, load the record its top selects ----
        unsigned long long old = 0ull;
        const bool hit = BITS != 0 && mode == E_CLAIM && ((*BITW(x) >> (x & 31)) & 1u);
        if (mode == E_CLAIM && !hit) old = atomicCAS(&SV(x).st, 0ull, mytag << K_BITS);
        else if (mode == E_CLAIM2) old = atomicCAS(&SV(x).st, cexp, (mytag << K_BITS) | (cexp & K_MASK));
        else if (mode == E_WAIT) old = ld_volatile(&SV(x).st);
        uint4 ri = make_uint4(0u, 0u, 0u, 0u);
        if (mode == E_START) ri = __ldg(rinfo + x);
        if (WGT && mode == E_THR) {
          // thresholds of a start vertex: high words of its B row
          const uint32_t m = xd > 13u ? 12u : (xd > 0u ? xd - 1u : 0u);
          for (uint32_t j = 0; j < m; ++j) cp_async4(thr_cur + j, (const uint32_t*)(Brow + xo + j) + 1);
          cp_async_commit();
        }
        const bool walk = (mode == E_POP) || (mode == E_RETRACE) || (mode == E_RELEASE);
        uint32_t nc = 0;
        if (walk) nc = LD_NXT(c);
        const bool topc = (mode == E_CLAIM && !hit) || (mode == E_CLAIM2) || (mode == E_TOP);
        bool nb = false;
        uint4 er = make_uint4((uint32_t)n, 0u, 0u, 0u);
        if (topc) {
          const uint32_t ks = mode == E_TOP ? kx : (mode == E_CLAIM2 ? (uint32_t)(cexp & K_MASK) : 0u);
          const uint4 o = philox4x32_10(ks, (uint32_t)x, tg, (uint32_t)a, p.key0, p.key1);
          const uint64_t u = stack_u53(o);
          const uint32_t uh = (uint32_t)(u >> 21);
          if (uh != xth) {
            nb = uh > xth;
          } else {
            const uint4 rx = __ldg(rinfo + x);
            nb = u >= ((uint64_t)rx.z | ((uint64_t)rx.w << 32));
          }
          if (nb) {
            uint32_t slot;
            if (!WGT) {
              slot = __umulhi(o.z, xd);
            } else {
              // first slot j with u < B_j; B_{d-1} = 2^53
              const uint32_t uh = (uint32_t)(u >> 32);
              const uint32_t m = xd > 13u ? 12u : xd - 1u;
              // (a loop of m trips: low-degree rows, the common case on road-like
              // graphs, skip the rest of the 12 words)
              slot = 0xffffffffu;
              for (uint32_t j = 0; j < m; ++j) {
                const uint32_t b = thr_cur[j];
                if (uh < b || (uh == b && u < __ldg(Brow + xo + j))) {
                  slot = j;
                  break;
                }
              }
              if (slot == 0xffffffffu) {
                if (xd - 1u > 12u) {
                  uint32_t lo = 12u, hi = xd - 1u;  // search B_12 .. B_{d-2}; hi = d - 1 means none
                  while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (u < __ldg(Brow + xo + mid)) hi = mid;
                    else lo = mid + 1u;
                  }
                  slot = lo;
                } else {
                  slot = xd - 1u;
                }
              }
            }
            const uint4* rec = edges + (size_t)(xo + slot) * (WGT ? 4 : 1);
            er = __ldg(rec);
            if (WGT) {
              cp_async16(thr_nxt, rec + 1);
              cp_async16(thr_nxt + 4, rec + 2);
              cp_async16(thr_nxt + 8, rec + 3);
              cp_async_commit();
            }
          }
        }

        // ---- consume ----
        bool finished = false;  // the path reached the tree or u*
        switch (mode) {
          case E_START: {  // row info of a restart vertex
            xo = ri.x;
            xd = ri.y;
            xth = thr_hi(ri);
            mode = WGT ? E_THR : E_CLAIM;
            break;
          }
          case E_THR: {  // thresholds of x copied: claim it next
            mode = E_CLAIM;
            break;
          }
          case E_CLAIM:
          case E_CLAIM2: {
            if (hit) {
              CNT(CNT_TREE_HIT);
              finished = true;
              break;
            }
            if (mode == E_CLAIM ? (old == 0ull) : (old == cexp)) {
              // x joins this walker's path with its top at entry kx
              CNT(CNT_CLAIM_OK);
              kx = mode == E_CLAIM ? 0u : (uint32_t)(cexp & K_MASK);
              if (kx >= (uint32_t)K_MASK - 1u) {
                // a pop while x is owned adds at most one more: keep k below 2^24
                atomicOr(p.err, ERR_OVERFLOW);
                ABORT_TREE();
                mode = E_DONE;
                break;
              }
              h = x;
              if (RINGP) {
                RING(len) = (uint32_t)x;
                ++len;
                if (len - rbase > PB) rbase = len - PB;
              } else {
                if (len < PB) sh_pb[len * W + me] = (uint32_t)x;
                ++len;
              }
              ++deps;
              ST_NXT(x, er.x);  // er.x = n when the entry selects u*
              if (!nb) {
                atomicAdd(p.R + (size_t)a * n + x, 1u);
                if (p.C != nullptr && kx == 0u) atomicAdd(p.C + (size_t)a * n + x, 1u);
                finished = true;
                fexit = true;
                break;
              }
              x = (int32_t)er.x;
              xo = er.y;
              xd = er.z;
              xth = er.w;
              cur ^= 1u;
              mode = E_CLAIM;
              if (EARLY_HIT(x)) {
                CNT(CNT_TREE_HIT);
                finished = true;
              }
              break;
            }
            if (mode == E_CLAIM2) {
              mode = E_CLAIM;  // the state changed under us: look again
              break;
            }
            if (old & IN_TREE) {
              CNT(CNT_TREE_HIT);
              finished = true;
              break;
            }
            const unsigned long long tag = (old >> K_BITS) & TAG_MASK;
            if (tag == 0ull) {
              cexp = old;  // free with k > 0
              mode = E_CLAIM2;
              break;
            }
            const uint32_t w = (uint32_t)(tag & EW_MASK);
            const uint32_t tgen = (uint32_t)(tag >> EW_BITS);
            if (w >= WT) {
              atomicOr(p.err, ERR_INVAL);
              ABORT_TREE();
              mode = E_DONE;
              break;
            }
            if (w == wid && tgen == gen) {
              // x closes a cycle on this walker's path: pop it.  When x is
              // among the last PB path vertices the cycle is in the ring and is
              // popped here (no loads); otherwise it is walked through nxt.
              kx = (uint32_t)(old & K_MASK);
              int32_t pos = -1;
              if (RINGP) {
#pragma unroll
                for (int i = 0; i < PB; ++i) {
                  const int32_t q = len - 1 - i;
                  if (pos < 0 && q >= rbase && RING(q) == (uint32_t)x) pos = q;
                }
              }
              if (RINGP && pos >= 0) {
                CNT(CNT_POP);
#pragma unroll
                for (int i = 1; i < PB; ++i) {
                  const int32_t q = pos + i;
                  if (q < len) {
                    ADD_ST(RING(q), 1ull - (mytag << K_BITS));
                    ++pops;
                  }
                }
                ADD_ST(x, 1ull);
                ++pops;
                ++kx;
                if (kx >= (uint32_t)K_MASK) {
                  atomicOr(p.err, ERR_OVERFLOW);
                  ABORT_TREE();
                  mode = E_DONE;
                  break;
                }
                len = pos + 1;
                h = x;
                mode = E_TOP;
                break;
              }
              c = x;
              rh = 0;  // vertices popped by the walk
              rskip = true;
              mode = E_POP;
              break;
            }
            // w finished that path (its flag is on its way) or gave x up after
            // our read: look again
            if (GEN_OF(w) != tgen) {
              CNT(CNT_CONFIRM);
              break;
            }
            if (h < 0 || wid < w) {
              CNT(CNT_SPIN);
              break;  // wait-die: wait
            }
            CNT(CNT_RELEASE);
            // die: give the path back without popping anything: the ring part
            // now, the older part by a walk from s (each vertex freed after its
            // nxt has been read)
            wtag = tag;
            if (RINGP) {
              const int32_t held = len - rbase;  // ring slots in use, in any order
#pragma unroll
              for (int i = 0; i < PB; ++i)
                if (((i - rbase) & (PB - 1)) < held) ADD_ST(sh_pb[i * W + me], 0ull - (mytag << K_BITS));
              if (rbase > 0) {
                c = s;
                rh = rbase;  // vertices left to free
                mode = E_RELEASE;
              } else if (!wdone && sh_ps[me] == NO_PARK) {
                // park the path and take other start vertices meanwhile
                sh_ps[me] = (uint32_t)s | PARK_FRESH;
                sh_px[me] = (uint32_t)x;
                sh_ptag[me] = wtag;
                mode = E_IDLE;
              } else {
                mode = E_WAIT;
              }
            } else {
              // prefix: free it now except the last entry, whose nxt the
              // release walk still reads
              const int nfree = len > PB ? PB - 1 : len;
              for (int i = 0; i < PB; ++i)
                if (i < nfree) ADD_ST(sh_pb[i * W + me], 0ull - (mytag << K_BITS));
              if (len > PB) {
                c = (int32_t)sh_pb[(PB - 1) * W + me];
                rh = h;  // the walk ends at the head
                mode = E_RELEASE;
              } else {
                mode = E_WAIT;
              }
            }
            h = -1;
            len = 0;
            rbase = 0;
            break;
          }
          case E_TOP: {  // top of the path head x at entry kx > 0 (after a pop)
            CNT(CNT_EDGE);
            ++deps;
            ST_NXT(x, er.x);
            if (!nb) {
              atomicAdd(p.R + (size_t)a * n + x, 1u);
              finished = true;  // kx > 0 here: the control variate counts entry 0 only
              fexit = true;
              break;
            }
            x = (int32_t)er.x;
            xo = er.y;
            xd = er.z;
            xth = er.w;
            cur ^= 1u;
            mode = E_CLAIM;
            if (EARLY_HIT(x)) {
              CNT(CNT_TREE_HIT);
              finished = true;
            }
            break;
          }
          case E_POP: {
            // cycle x -> ... -> h -> x: free every vertex but x at its next entry
            CNT(CNT_POP);
            if (!rskip) {
              if (nxt_read(nc)) ADD_ST(c, 1ull - (mytag << K_BITS));
              ++pops;
              if (RINGP || ROOTS) ++rh;
            }
            rskip = false;
            c = (int32_t)nc;
            if (c == x) {
              ADD_ST(x, 1ull);
              ++pops;
              ++kx;
              if (kx >= (uint32_t)K_MASK) {
                atomicOr(p.err, ERR_OVERFLOW);
                ABORT_TREE();
                mode = E_DONE;
                break;
              }
              if (RINGP) {
                // the path now ends at x, whose position is below the ring
                len -= rh;
                rbase = len - 1;
                RING(rbase) = (uint32_t)x;
              } else {
                // the path now ends at x (with ROOTS the length stays exact
                // when x lies beyond the prefix: depths count along the path)
                int32_t pos = len;
                for (int i = 0; i < PB; ++i)
                  if (i < len && sh_pb[i * W + me] == (uint32_t)x) pos = i;
                if (pos < PB) len = pos + 1;
                else if (ROOTS) len -= rh;
              }
              h = x;
              mode = E_TOP;
            }
            break;
          }
          case E_RETRACE: {
            if (!rskip) {
              if (ROOTS) {
                RD[c - base] = rd_pack(froot, fdl + (flen - 1 - fpos));
                __threadfence_block();  // every reader is in this CTA (no clusters)
              }
              if (BITS != 0) atomicOr((uint32_t*)BITW(c), 1u << (c & 31));
              else OR_ST(c, IN_TREE);
            }
            rskip = false;
            if (RINGP ? --rh == 0 : c == rh) {
              mode = E_IDLE;
            } else {
              c = (int32_t)nc;
              ++fpos;
            }
            break;
          }
          case E_RELEASE: {
            if (nxt_read(nc)) ADD_ST(c, 0ull - (mytag << K_BITS));
            if (RINGP ? --rh == 0 : c == rh) {
              if (RINGP && !wdone && sh_ps[me] == NO_PARK) {  // park (see the release above)
                sh_ps[me] = (uint32_t)s | PARK_FRESH;
                sh_px[me] = (uint32_t)x;
                sh_ptag[me] = wtag;
                mode = E_IDLE;
              } else {
                mode = E_WAIT;
              }
            } else {
              c = (int32_t)nc;
            }
            break;
          }
          case E_WAIT: {
            CNT(CNT_WAIT);
            const uint32_t ww = (uint32_t)(wtag & EW_MASK);
            const bool parked = RINGP && sh_ps[me] == (uint32_t)s;  // the wait of a parked path
            if ((old >> K_BITS) == wtag && GEN_OF(ww) == (uint32_t)(wtag >> EW_BITS)) {
              if (parked && !wdone) {  // still in the way: other start vertices first
                sh_ps[me] = (uint32_t)s | PARK_FRESH;
                mode = E_IDLE;
              }
              break;
            }
            if (parked) sh_ps[me] = NO_PARK;
            x = s;
            mode = E_START;
            break;
          }
          default:
            break;
        }

        if (finished) {
          // the path s -> ... -> h joins the tree: bump the generation, then flag
          // the ring part and walk the older part from s
          if (len > 0) {
            if (!CL && p.ramp_q != 0u) atomicAdd(&sh_tsize, (uint32_t)len);
            ++gen;
            if (gen >= GEN_LIMIT) {  // the tag has 26 generation bits
              atomicOr(p.err, ERR_OVERFLOW);
              ABORT_TREE();
            }
            sh_gen[me] = gen;
            // ring: slots in use in any order; prefix: the first min(len, PB)
            const int32_t held = RINGP ? len - rbase : len;
            if (ROOTS) {
              // root and depth base: the head's own (exit to u*) or x's, read
              // after x was seen in the tree
              if (fexit) {
                froot = h;
                fdl = 0;
              } else {
                const unsigned long long rx = *(volatile unsigned long long*)&RD[x - base];
                froot = (int32_t)(uint32_t)rx;
                fdl = (int32_t)(uint32_t)(rx >> 32) + 1;
              }
              flen = len;
#pragma unroll
              for (int i = 0; i < PB; ++i) {
                const int32_t q = RINGP ? rbase + ((i - rbase) & (PB - 1)) : i;  // path position of slot i
                if (q - (RINGP ? rbase : 0) < held) {
                  const uint32_t v = sh_pb[i * W + me];
                  RD[v - base] = rd_pack(froot, fdl + (len - 1 - q));
                }
              }
              __threadfence_block();
              fpos = RINGP ? 0 : PB - 1;  // where the walk from s (or the prefix's end) starts
            }
#pragma unroll
            for (int i = 0; i < PB; ++i) {
              if ((RINGP ? ((i - rbase) & (PB - 1)) : i) < held) {
                const uint32_t v = sh_pb[i * W + me];
                if (BITS != 0) atomicOr((uint32_t*)BITW(v), 1u << (v & 31));
                else OR_ST(v, IN_TREE);
              }
            }
            if (RINGP && rbase > 0) {
              c = s;
              rh = rbase;  // vertices left to flag
              rskip = false;
              mode = E_RETRACE;
            } else if (!RINGP && len > PB) {
              c = (int32_t)sh_pb[(PB - 1) * W + me];  // flagged above; the walk ends at the head
              rh = h;
              rskip = true;
              mode = E_RETRACE;
            } else {
              mode = E_IDLE;
            }
          } else {
            mode = E_IDLE;
          }
          h = -1;
          len = 0;
          rbase = 0;
          fexit = false;
        }
      }

      if (refill) {
        // the new window: slots whose vertex is not in the tree yet
        cp_async_wait_all();
        __syncwarp();
        bool cand = wok;
        if (wok) {
          if (BITS != 0) {
            const uint32_t v = sh_wv[lane];
            cand = ((*BITW(v) >> (v & 31)) & 1u) == 0u;
          } else {
            cand = (sh_wst[lane].y & (uint32_t)(IN_TREE >> 32)) == 0u;
          }
        }
        // compact the candidates to the front of the window, in place: a lane
        // writes slot pos <= lane, which another lane reads as its own, so every
        // read comes before every write (a vote orders no memory accesses
        // between lanes; only __syncwarp does: without it a lane's read was
        // moved after another lane's write, and start vertices were lost)
        uint4 wr = make_uint4(0u, 0u, 0u, 0u);
        uint32_t wv = 0;
        if (cand) {
          wr = sh_wri[lane];
          wv = sh_wv[lane];
        }
        const unsigned cm = __ballot_sync(FULL, cand);
        __syncwarp();
        if (cand) {
          const uint32_t pos = (uint32_t)__popc(cm & lt_mask);
          sh_wri[pos] = wr;
          sh_wv[pos] = wv;
        }
        __syncwarp();
        whead = 0;
        wcnt = (uint32_t)__popc(cm);
        if (wb + 32u >= (uint32_t)nl) wdone = true;
      }
    }

    cp_async_wait_all();  // no copy of this tree may land in the next one's buffers
    if (CL) {  // the tree's totals are kept by rank 0
      atomicAdd(cg::this_cluster().map_shared_rank(&sh_pops, 0u), (unsigned long long)pops);
      atomicAdd(cg::this_cluster().map_shared_rank(&sh_deps, 0u), (unsigned long long)deps);
    } else {
      atomicAdd(&sh_pops, (unsigned long long)pops);
      atomicAdd(&sh_deps, (unsigned long long)deps);
    }
#if FC_WILSON_COUNTERS
#pragma unroll
    for (int q = 0; q < N_CNT; ++q) {
      unsigned long long vq = cnt[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vq += __shfl_xor_sync(FULL, vq, o);
      if (lane == 0 && vq) atomicAdd(&p.stats[2 + q], vq);
    }
#endif
    if (CL) cg::this_cluster().sync();  // every walker of the tree has finished
    else __syncthreads();
    const size_t item = p.num_graphs > 0 ? (size_t)gi * (size_t)p.tau + (size_t)tloc : (size_t)tree;
    if (p.parents != nullptr) {
      int32_t* par = p.parents + (p.num_graphs > 0 ? (size_t)tloc : (size_t)tree) * n + base;
      for (int32_t v = (int32_t)wid; v < nl; v += (int32_t)WT) par[v] = (int32_t)S[v].nxt;
    }
    if (ROOTS) {  // the forest, copied out coalesced
      const size_t row = (p.num_graphs > 0 ? (size_t)tloc : (size_t)tree) * (size_t)n + (size_t)base;
      for (int32_t v = (int32_t)wid; v < nl; v += (int32_t)WT) {
        const unsigned long long pk = RD[v];
        if (p.roots) p.roots[row + v] = (int32_t)(uint32_t)pk;
        if (p.depths) p.depths[row + v] = (int32_t)(uint32_t)(pk >> 32);
      }
    }
    if (p.visits != nullptr) {  // departures from v = its popped stack entries + the tree edge's
      unsigned long long* vis = p.visits + (size_t)a * n + base;
      for (int32_t v = (int32_t)wid; v < nl; v += (int32_t)WT) atomicAdd(&vis[v], (S[v].st & K_MASK) + 1ull);
    }
    if (me == 0 && rank == 0) {
      if (p.steps != nullptr) p.steps[item] = (uint64_t)nl + sh_pops;
      if (p.item_ns != nullptr) p.item_ns[item] = global_ns();
      atomicAdd(&p.stats[0], sh_pops);
      atomicAdd(&p.stats[1], sh_deps);
    }
    if (CL) cg::this_cluster().sync();  // parents read before the state is cleared again
    else __syncthreads();
  }
#undef RING
#undef SV
#undef REMOTE
#undef BITW
#undef EARLY_HIT
#undef GEN_OF
#undef ABORT_TREE
#undef ADD_ST
#undef OR_ST
#undef LD_NXT
#undef ST_NXT
}

template <int BITS, bool WGT, bool RINGP, bool CL>
static WilsonFn edge_fn_regs(int regs) {
  return regs <= 48 ? k_wilson_edge<BITS, WGT, RINGP, CL, 48, false> : k_wilson_edge<BITS, WGT, RINGP, CL, 64, false>;
}

template <int BITS, bool WGT, bool CL>
static WilsonFn edge_fn_ring(bool ring, int regs) {
  return ring ? edge_fn_regs<BITS, WGT, true, CL>(regs) : edge_fn_regs<BITS, WGT, false, CL>(regs);
}

template <int BITS, bool CL>
static WilsonFn edge_fn_wgt(bool wgt, bool ring, int regs) {
  return wgt ? edge_fn_ring<BITS, true, CL>(ring, regs) : edge_fn_ring<BITS, false, CL>(ring, regs);
}

// forest-root variants: 64 registers, no clusters
template <int BITS, bool WGT>
static WilsonFn edge_fn_roots(bool ring) {
  return ring ? k_wilson_edge<BITS, WGT, true, false, 64, true> : k_wilson_edge<BITS, WGT, false, false, 64, true>;
}

WilsonFn wilson_edge_fn(int bits, bool wgt, bool ring, bool cl, int regs, bool roots) {
  if (roots) {
    if (bits == 1) return wgt ? edge_fn_roots<1, true>(ring) : edge_fn_roots<1, false>(ring);
    if (bits == 2) return wgt ? edge_fn_roots<2, true>(ring) : edge_fn_roots<2, false>(ring);
    return wgt ? edge_fn_roots<0, true>(ring) : edge_fn_roots<0, false>(ring);
  }
  if (cl) return bits == 1 ? edge_fn_wgt<1, true>(wgt, ring, regs) : edge_fn_wgt<0, true>(wgt, ring, regs);
  if (bits == 1) return edge_fn_wgt<1, false>(wgt, ring, regs);
  if (bits == 2) return edge_fn_wgt<2, false>(wgt, ring, regs);
  return edge_fn_wgt<0, false>(wgt, ring, regs);
}

size_t wilson_edge_smem(int W, int32_t n, int bits, bool wgt, int C, bool ring) {
  // the start window keeps state records only when membership is a state flag;
  // ring variants keep a parked path per walker
  const size_t base = (((size_t)W * 4 * (1 + PB) + 15) & ~(size_t)15) +
                      (size_t)W * (16 + (bits == 0 ? 16 : 0) + 4 + (ring ? 16 : 0));
  const size_t words = ((size_t)n + 31) / 32;
  return ((base + 15) & ~(size_t)15) + (wgt ? (size_t)W * 2 * 12 * 4 : 0) +
         (bits == 1 ? ((words + (size_t)C - 1) / (size_t)C) * 4 : 0);
}

}  // namespace fcx
