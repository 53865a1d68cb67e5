// Uniform spanning trees of G* rooted at u* (Algorithm 2, App. B) for the
// sampling loop of Algorithm 1, and the u*-edge counts of Prop. 1.
//
// Design (GB300): a persistent kernel, one CTA per tree at a time, W walkers
// (threads) per tree running Wilson walks from different start vertices at
// once.  The random choices come from "random stacks" (stack entry k of vertex
// v in tree t = Philox4x32-10 of (k, v, t, alpha index)); with stacks fixed,
// Wilson's algorithm is cycle popping (Propp-Wilson), whose result -- the tree
// and the number of pops of every vertex -- does not depend on the order in
// which cycles are popped.  Each walker only ever pops cycles that lie on its
// own path and only joins the tree through vertices already in it, so every
// interleaving is a valid cycle-popping order and the trees are bit-identical
// to the sequential sampler's.
//
// Per-tree state, one 16-byte record per vertex (global memory, or shared
// memory for small graphs):
//   st  bits  0..23  k = stack entries of v popped so far (the current top is
//                     entry k)
//       bits 24..63  tag: 0 = free; otherwise (gen << 10) | walker -- v lies on
//                     the path that walker had in generation gen
//   nxt the vertex selected by v's current top (valid while v is owned or in
//       the tree)
// A vertex is in the tree iff its tag names a generation that its walker has
// already finished (walkers bump their generation, in shared memory, when a
// path reaches the tree), so joining the tree needs no retrace of the path.
// Conflicts between walkers of one tree use wait-die on walker ids: a walker
// waits for a higher-numbered walker, and releases its whole path (without
// popping anything: the stacks stay as they were) when blocked by a
// lower-numbered one; a walker holding no vertex may always wait.  Waits thus
// only point from lower to higher walker ids and cannot form a cycle.
#include <algorithm>

#include "fc_wilson_common.cuh"

namespace fcx {

// Record msg as the last error and return FC_EINVAL.
static inline fc_status invalid(const char* msg) {
  set_error(msg);
  return FC_EINVAL;
}

enum { P_IDLE = 0, P_CHECK, P_CLAIM, P_CLAIM2, P_EDGE, P_NEXT, P_POP, P_RETRACE, P_RELEASE, P_WAIT,
       P_DONE };
constexpr uint32_t NO_START = 0xffffffffu;

// One loop iteration = at most one dependent round trip to memory per walker:
// the memory operations of the iteration are issued (predicated by the
// walker's mode) before results are consumed, so the 32 walkers of a warp
// overlap their waits whatever mix of modes they are in.  A departure takes
// two iterations: CHECK (in-tree bit + row info, both L2-resident) and CLAIM
// (CAS on the 16-byte state, with the stack entry for k = 0 computed
// speculatively and its CSR target loaded alongside).  Tree membership lives
// only in the bitmap, so tree hits and the marking of finished paths never
// touch the state array.
template <bool SMEM, int MAXREG>
__global__ void __launch_bounds__(1024) __maxnreg__(MAXREG) k_wilson(WParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long sh_tree, sh_pops, sh_deps;
  __shared__ uint32_t sh_next;
  __shared__ volatile uint32_t sh_abort;
  const int me = threadIdx.x;
  const int W = blockDim.x;
  const int lane = me & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  volatile uint32_t* sh_gen = (volatile uint32_t*)smem_raw;
  uint32_t* sh_pb = (uint32_t*)(smem_raw + (size_t)W * 4);  // [PB][W] path prefix of each walker
  const int32_t n = p.n;  // u* = n (global numbering)
  const int32_t words = p.words;
  if (p.t0_ns != nullptr && threadIdx.x == 0) atomicMin(p.t0_ns, global_ns());
  // Tree-major state: each CTA's trees use their own contiguous column.  (A
  // vertex-major layout, which lets trees share lines at common start
  // vertices, measured slower: atomics from many SMs then meet on one line.)
  VState* S;
  uint32_t* bits;
  if (SMEM) {
    unsigned char* sbase = smem_raw + (((size_t)W * 4 * (1 + PB) + 15) & ~(size_t)15);
    S = (VState*)sbase;
    bits = (uint32_t*)(sbase + (size_t)p.nmax * sizeof(VState));
  } else {
    S = p.gstate + (size_t)blockIdx.x * p.nmax;
    bits = p.gbits + (size_t)blockIdx.x * words;
  }
#define SV(v) S[(v) - base]
#define BWV(v) bits[((v) - base) >> 5]
#define BITV(v) (1u << (((v) - base) & 31))
#define LD_BITS(v) ld_volatile32(&BWV(v))
#define OR_BITS(v) ((void)atomicOr(&BWV(v), BITV(v)))
#define CAS_ST(v, cmp, val) atomicCAS(&SV(v).st, (cmp), (val))
#define ADD_ST(v, d) ((void)atomicAdd(&SV(v).st, (d)))
#define LD_NXT(v) SV(v).nxt
#define ST_NXT(v, t) ((void)(SV(v).nxt = (t)))
#define LD_RINFO(v) __ldg(rinfo + (v))
#define LD_COL(e) __ldg(p.colidx + (e))
  bool first_tree = true;
  const int64_t total = (int64_t)(p.num_graphs > 0 ? p.num_graphs : p.n_alpha) * p.tau;

  for (;;) {
    if (me == 0) sh_tree = atomicAdd(p.counter, 1ull);
    __syncthreads();
    const unsigned long long tree = sh_tree;
    if ((int64_t)tree >= total || *(volatile uint32_t*)p.err != 0u) break;
    // item -> (alpha index or graph, tree); the tree's vertices are [base, base + nl)
    const unsigned long long tq = tree / (unsigned long long)p.tau;
    const int64_t tloc = (int64_t)(tree % (unsigned long long)p.tau);
    int a = (int)tq;
    int32_t base = 0, nl = n, gi = 0;
    if (p.num_graphs > 0) {
      gi = p.gorder[tq];
      a = 0;
      base = (int32_t)p.voff[gi];
      nl = (int32_t)(p.voff[gi + 1] - p.voff[gi]);
    }
    const uint32_t tg = (uint32_t)(p.tree_offset + tloc);
    if (!(first_tree && p.pre_cleared)) {
      for (int32_t v = me; v < nl; v += W) reinterpret_cast<uint4&>(S[v]) = make_uint4(0u, 0u, 0u, 0u);
      for (int32_t q = me; q < ((nl + 31) >> 5); q += W) bits[q] = 0u;
    }
    first_tree = false;
    sh_gen[me] = 1u;
    if (me == 0) {
      sh_next = 0;
      sh_abort = 0;
      sh_pops = 0;
      sh_deps = 0;
    }
    __syncthreads();

    const uint4* __restrict__ rinfo = p.rowinfo + (size_t)a * n;

    int mode = P_IDLE;
    int32_t x = 0, h = -1, c = 0, rh = 0, s = 0;
    int32_t len = 0;           // vertices on the current path
    bool rskip = false;        // the first walk step only loads (vertex already handled)
    uint32_t sni = NO_START;
    int32_t sn = -1;
    uint4 xr = make_uint4(0u, 0u, 0u, 0u);  // row info of x
    uint32_t enext = 0;        // CSR entry of h's selected neighbour (P_NEXT)
    bool need = true;
    uint32_t gen = 1, kx = 0, iters = 0, pops = 0, deps = 0;
    unsigned long long wtag = 0, cexp = 0;
#if FC_WILSON_COUNTERS
    uint32_t cnt[N_CNT];
#pragma unroll
    for (int q = 0; q < N_CNT; ++q) cnt[q] = 0;
#endif

    while (true) {
      __syncwarp();
      const bool fin = (mode == P_DONE) || (sh_abort != 0u);
      if (__all_sync(FULL, fin)) break;
      const unsigned want = __ballot_sync(FULL, need && !fin);
      if (want) {
        const int leader = __ffs(want) - 1;
        uint32_t ibase = 0;
        if (lane == leader) ibase = atomicAdd(&sh_next, (uint32_t)__popc(want));
        ibase = __shfl_sync(FULL, ibase, leader);
        if (need && !fin) {
          sni = ibase + __popc(want & lt_mask);
          const uint32_t ix = p.descending ? (uint32_t)nl - 1u - sni : sni;
          sn = sni < (uint32_t)nl ? (p.id_order ? base + (int32_t)ix : __ldg(p.order + base + ix)) : -1;
          need = false;
        }
      }
      if (fin) {
        CNT(CNT_IDLE_LANE);
        continue;
      }
      CNT(CNT_ITER);
      if (++iters > p.max_iters) {
        atomicOr(p.err, ERR_TIMEOUT);
        sh_abort = 1u;
        mode = P_DONE;
        continue;
      }
      if (mode == P_IDLE) {
        if (sn < 0) {
          mode = P_DONE;
          continue;
        }
        if (sn < base || sn >= base + nl) {  // start order must stay inside the tree's vertex range
          atomicOr(p.err, ERR_INVAL);
          sh_abort = 1u;
          mode = P_DONE;
          continue;
        }
        s = sn;
        x = s;
        h = -1;
        len = 0;
        mode = P_CHECK;
        need = true;
      }
      const unsigned long long mytag = ((unsigned long long)gen << W_BITS) | (unsigned)me;

      // ---- issue ----
      // STEP (= CHECK then CLAIM of x within one iteration): the in-tree bit
      // and row info of x come from L2; only if the bit is clear does the
      // walker touch the 16-byte state (CAS), with the stack entry for k = 0
      // computed and its CSR target loaded speculatively alongside.
      bool hit = false;
      if (mode == P_CHECK) {
        const uint32_t bw = LD_BITS(x);
        xr = LD_RINFO(x);
        hit = (bw & BITV(x)) != 0u;
        if (!hit) mode = P_CLAIM;
      }
      unsigned long long old = 0ull;
      if (mode == P_CLAIM) old = CAS_ST(x, 0ull, mytag << K_BITS);
      else if (mode == P_CLAIM2) old = CAS_ST(x, cexp, (mytag << K_BITS) | (cexp & K_MASK));
      else if (mode == P_WAIT) old = ld_volatile(&SV(x).st);
      const bool walk = (mode == P_POP) || (mode == P_RETRACE) || (mode == P_RELEASE);
      uint32_t nc = 0;
      if (walk) nc = LD_NXT(c);
      // the stack entry: k = 0 speculatively while claiming, kx when computing a top
      const bool topc = (mode == P_CLAIM) || (mode == P_EDGE);
      uint32_t e = 0;
      bool nb = false;
      if (topc) {
        const uint4 o = philox4x32_10(mode == P_EDGE ? kx : 0u, (uint32_t)x, tg, (uint32_t)a, p.key0, p.key1);
        nb = select_edge(p, a, xr, o, &e);
      }
      int32_t t = n;
      if (topc && nb) t = LD_COL(e);
      else if (mode == P_NEXT) t = LD_COL(enext);

      // ---- consume ----
      bool finished = false;  // the path reached the tree or u*
      switch (mode) {
        case P_CHECK: {  // x is in the tree
          CNT(CNT_TREE_HIT);
          finished = true;
          break;
        }
        case P_CLAIM:
        case P_CLAIM2: {
          if (mode == P_CLAIM ? (old == 0ull) : (old == cexp)) {
            // x joins this walker's path
            h = x;
            if (len < PB) sh_pb[len * W + me] = (uint32_t)x;
            ++len;
            if (mode == P_CLAIM2) {
              kx = (uint32_t)(cexp & K_MASK);
              if (kx >= (uint32_t)K_MASK - 1u) {
                atomicOr(p.err, ERR_OVERFLOW);
                sh_abort = 1u;
                mode = P_DONE;
                break;
              }
              mode = P_EDGE;  // its top at entry k > 0 is computed next iteration
              break;
            }
            CNT(CNT_CLAIM_OK);
            ++deps;
            ST_NXT(h, (uint32_t)t);
            if (!nb) {
              atomicAdd(p.R + (size_t)a * n + h, 1u);
              if (p.C != nullptr) atomicAdd(p.C + (size_t)a * n + h, 1u);
              finished = true;
              break;
            }
            x = t;
            mode = P_CHECK;
            break;
          }
          if (mode == P_CLAIM2) {
            mode = P_CHECK;  // the state changed under us: look again
            break;
          }
          const unsigned long long tag = old >> K_BITS;
          if (tag == 0ull) {
            cexp = old;  // free with k > 0
            mode = P_CLAIM2;
            break;
          }
          const uint32_t w = (uint32_t)(tag & ((1u << W_BITS) - 1));
          const uint32_t tgen = (uint32_t)(tag >> W_BITS);
          if (w >= (uint32_t)W) {
            atomicOr(p.err, ERR_INVAL);
            sh_abort = 1u;
            mode = P_DONE;
            break;
          }
          if (w == (uint32_t)me && tgen == gen) {
            // x closes a cycle on this walker's path: pop it
            kx = (uint32_t)(old & K_MASK);
            c = x;
            rskip = true;
            mode = P_POP;
            break;
          }
          if (sh_gen[w] != tgen) {
            // w finished that path (x is being marked in the tree) or gave x up
            // after our read: look again, starting with the bit
            CNT(CNT_SPIN);
            mode = P_CHECK;
            break;
          }
          if (h < 0 || (uint32_t)me < w) {
            CNT(CNT_SPIN);  // wait-die: wait
            break;
          }
          // die: give the path back without popping anything; vertices whose
          // nxt the release walk still needs are freed only after it is read
          CNT(CNT_RELEASE);
          wtag = tag;
          const int nfree = len > PB ? PB - 1 : len;
          for (int i = 0; i < PB; ++i)
            if (i < nfree) ADD_ST(sh_pb[i * W + me], 0ull - (mytag << K_BITS));
          if (len > PB) {
            c = (int32_t)sh_pb[(PB - 1) * W + me];
            rh = h;
            rskip = false;
            mode = P_RELEASE;
          } else {
            mode = P_WAIT;
          }
          h = -1;
          len = 0;
          break;
        }
        case P_EDGE: {
          CNT(CNT_EDGE);
          ++deps;
          ST_NXT(h, (uint32_t)t);
          if (!nb) {
            atomicAdd(p.R + (size_t)a * n + h, 1u);
            if (p.C != nullptr && kx == 0u) atomicAdd(p.C + (size_t)a * n + h, 1u);
            finished = true;
            break;
          }
          x = t;
          mode = P_CHECK;
          break;
        }
        case P_POP: {
          // cycle x -> ... -> h -> x: free every vertex but x at its next entry
          CNT(CNT_POP);
          if (!rskip) {
            if (nxt_read(nc)) ADD_ST(c, 1ull - (mytag << K_BITS));
            ++pops;
          }
          rskip = false;
          c = (int32_t)nc;
          if (c == x) {
            ADD_ST(x, 1ull);
            ++pops;
            ++kx;
            if (kx >= (uint32_t)K_MASK) {
              atomicOr(p.err, ERR_OVERFLOW);
              sh_abort = 1u;
              mode = P_DONE;
              break;
            }
            // the path now ends at x
            int32_t pos = len;
            for (int i = 0; i < PB; ++i)
              if (i < len && sh_pb[i * W + me] == (uint32_t)x) pos = i;
            if (pos < PB) len = pos + 1;
            h = x;
            mode = P_EDGE;
          }
          break;
        }
        case P_RETRACE: {
          if (!rskip) OR_BITS(c);
          rskip = false;
          if (c == rh) mode = P_IDLE;
          else c = (int32_t)nc;
          break;
        }
        case P_RELEASE: {
          if (nxt_read(nc)) ADD_ST(c, 0ull - (mytag << K_BITS));
          if (c == rh) mode = P_WAIT;
          else c = (int32_t)nc;
          break;
        }
        case P_WAIT: {
          CNT(CNT_WAIT);
          const uint32_t ww = (uint32_t)(wtag & ((1u << W_BITS) - 1));
          if ((old >> K_BITS) == wtag && sh_gen[ww] == (uint32_t)(wtag >> W_BITS)) break;
          x = s;
          mode = P_CHECK;
          break;
        }
        default:
          break;
      }

      if (finished) {
        // the path s -> ... -> h joins the tree: bump the generation (walkers
        // that meet the path from now on re-check the bit instead of dying),
        // then set the bits of the remembered prefix and walk the rest
        if (len > 0) {
          __threadfence_block();
          ++gen;
          sh_gen[me] = gen;
          for (int i = 0; i < PB; ++i)
            if (i < len) {
              const uint32_t v = sh_pb[i * W + me];
              OR_BITS(v);
            }
          if (len > PB) {
            c = (int32_t)sh_pb[(PB - 1) * W + me];
            rh = h;
            rskip = true;
            mode = P_RETRACE;
          } else {
            mode = P_IDLE;
          }
        } else {
          mode = P_IDLE;
        }
        h = -1;
        len = 0;
      }
    }

    atomicAdd(&sh_pops, (unsigned long long)pops);
    atomicAdd(&sh_deps, (unsigned long long)deps);
#if FC_WILSON_COUNTERS
#pragma unroll
    for (int q = 0; q < N_CNT; ++q) {
      unsigned long long vq = cnt[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vq += __shfl_xor_sync(FULL, vq, o);
      if (lane == 0 && vq) atomicAdd(&p.stats[2 + q], vq);
    }
#endif
    __syncthreads();
    const size_t item = (size_t)(p.num_graphs > 0 ? gi : a) * (size_t)p.tau + (size_t)tloc;
    if (p.parents != nullptr) {
      int32_t* par = p.parents + (p.num_graphs > 0 ? (size_t)tloc : (size_t)tree) * n + base;
      for (int32_t v = me; v < nl; v += W) par[v] = (int32_t)S[v].nxt;
    }
    if (p.visits != nullptr) {  // departures from v = its popped stack entries + the tree edge's
      unsigned long long* vis = p.visits + (size_t)a * n + base;
      for (int32_t v = me; v < nl; v += W) atomicAdd(&vis[v], (S[v].st & K_MASK) + 1ull);
    }
    if (me == 0) {
      if (p.steps != nullptr) p.steps[item] = (uint64_t)nl + sh_pops;
      if (p.item_ns != nullptr) p.item_ns[item] = global_ns();
      atomicAdd(&p.stats[0], sh_pops);
      atomicAdd(&p.stats[1], sh_deps);
    }
    __syncthreads();
  }
}

#undef SV
#undef BWV
#undef BITV
#undef LD_BITS
#undef OR_BITS
#undef CAS_ST
#undef ADD_ST
#undef LD_NXT
#undef ST_NXT
#undef LD_RINFO
#undef LD_COL

__global__ void k_stack_entries(WParams p, int a, uint32_t tg, int64_t count, const int32_t* __restrict__ verts,
                                const uint32_t* __restrict__ ks, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int32_t v = verts[i];
  if (v < 0 || v >= p.n) {
    out[i] = -1;
    atomicOr(p.err, ERR_INVAL);
    return;
  }
  const uint4 ri = p.rowinfo[(size_t)a * p.n + v];
  const uint4 o = philox4x32_10(ks[i], (uint32_t)v, tg, (uint32_t)a, p.key0, p.key1);
  uint32_t e = 0;
  out[i] = select_edge(p, a, ri, o, &e) ? p.colidx[e] : p.n;
}

static size_t smem_bytes(int W, int32_t n, bool smem) {
  const size_t gen = ((size_t)W * 4 * (1 + PB) + 15) & ~(size_t)15;
  const size_t words = ((size_t)n + 31) / 32;
  return smem ? gen + (size_t)n * sizeof(VState) + words * 4 : gen;
}

static WilsonFn wilson_fn(bool smem, int regs) {
  if (smem) {
    if (regs == 32) return k_wilson<true, 32>;
    if (regs == 40) return k_wilson<true, 40>;
    return k_wilson<true, 64>;
  }
  if (regs == 32) return k_wilson<false, 32>;
  if (regs == 40) return k_wilson<false, 40>;
  return k_wilson<false, 64>;
}

constexpr size_t SBITS_CARVEOUT = 196 * 1024 - 1024 - 256;  // minus the per-CTA reserve and static shared memory

struct Shape {
  int W = 0;
  int regs = 64;
  int per_sm = 0;
  int64_t slots = 0;  // trees that can be in flight at once
};

// Launch shape: the walker count and register variant with the most walkers
// resident, weighted by how full the waves of trees are (a last wave that is
// mostly empty costs about as much as a full one).  Walkers per tree are
// capped at n/8.
static fc_status choose_shape(const fc_graph* g, int32_t n, int64_t total, bool smem, bool edge, int bits,
                              bool ring, int cl, int nsm, int smem_optin, Shape* out) {
  const bool sbits = bits == 1;
  // walks on G with one exit (fc_build_rooted) are long and cross each other:
  // measured on GB300 (BA n = 2^20 rooted at its hub, 256 trees), walkers
  // that release their paths under wait-die repeat 2.3x the departures at
  // 1024 walkers per tree and 1.03x at 128, which ran 2.7x faster
  const int wcap = std::max(32, std::min(g->root >= 0 ? 128 : 1024, (int)((n / 8) & ~31)));
  // measured on GB300 (BA n = 2^20, tau = 1024): the 40-register variant is
  // fastest; graphs with long walks prefer more walkers per tree, which the
  // score below already favours
  // (edge-record kernel: the 64-register variants; its 48-register ones spill,
  // the weighted ones heavily, and measured up to 2x slower)
  const int regs_list[2] = {edge ? 64 : 40, 64};
  double best = -1.0;
  for (int ri = 0; ri < (edge ? 1 : 2); ++ri) {
    int regs = g->regs > 0 ? g->regs : regs_list[ri];
    if (g->regs > 0 && ri > 0) break;
    if (!edge && regs == 48) regs = 40;
    if (edge && regs < 48) regs = 48;
    const WilsonFn fn = edge ? wilson_edge_fn(bits, g->weighted, ring, cl > 1, regs) : wilson_fn(smem, regs);
    for (int W = (g->walkers > 0 ? g->walkers : wcap); W >= 32; W -= 32) {
      const size_t shb = edge ? wilson_edge_smem(W, n, bits, g->weighted, cl, ring) : smem_bytes(W, n, smem);
      if (shb + 64 > (size_t)smem_optin) {
        if (g->walkers > 0) break;
        continue;
      }
      // measured on GB300 (BA n = 2^20): with the shared-memory bitmap, a CTA
      // that needs more than the 196 KB shared-memory carveout step runs about
      // 20% slower than one just below it (the L1 left for register spills
      // shrinks); automatic shapes stay below the step when they can
      if (sbits && g->walkers == 0 && shb > SBITS_CARVEOUT &&
          wilson_edge_smem(32, n, 1, g->weighted, cl, ring) <= SBITS_CARVEOUT)
        continue;
      if (edge) FC_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
      if (smem) FC_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
      int per_sm = 0;
      FC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, W, shb));
      int64_t slots = (int64_t)per_sm * nsm / cl;  // trees in flight
      if (cl > 1 && per_sm > 0) {
        // clusters are placed within a GPC: ask how many fit at once
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(cl * nsm));
        cfg.blockDim = dim3((unsigned)W);
        cfg.dynamicSmemBytes = shb;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int resident = 0;
        FC_CK(cudaOccupancyMaxActiveClusters(&resident, fn, &cfg));
        slots = resident;
      }
      if (per_sm > 0 && slots > 0) {
        const int64_t waves = (total + slots - 1) / slots;
        // walkers resident, times the average fill of the waves
        const double score = (double)W * (double)std::min<int64_t>(total, slots) * (double)total /
                             ((double)waves * (double)slots);
        if (score > best * 1.0001) {
          best = score;
          out->W = W;
          out->regs = regs;
          out->per_sm = per_sm;
          out->slots = slots;
        }
      }
      if (g->walkers > 0) break;
    }
  }
  if (out->W == 0) {
    set_error("fc_sample_usts: launch shape does not fit on an SM");
    return FC_EINVAL;
  }
  return FC_OK;
}

}  // namespace fcx

using namespace fcx;

static fc_status sample_impl(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R, uint32_t* C,
                             int32_t* parents, uint64_t* visits, uint64_t max_steps_per_tree, uint64_t* steps_out,
                             void* stream, bool sync, int32_t* roots = nullptr, int32_t* depths = nullptr);

extern "C" fc_status fc_sample_usts(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                                    uint32_t* C, int32_t* parents, uint64_t max_steps_per_tree,
                                    uint64_t* steps_out, void* stream) {
  return sample_impl(g, seed, tau, tree_offset, R, C, parents, nullptr, max_steps_per_tree, steps_out, stream, true);
}

extern "C" fc_status fc_sample_usts_forest(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                                           uint32_t* C, int32_t* parents, int32_t* roots, int32_t* depths,
                                           uint64_t* visits, uint64_t max_steps_per_tree, uint64_t* steps_out,
                                           void* stream) {
  return sample_impl(g, seed, tau, tree_offset, R, C, parents, visits, max_steps_per_tree, steps_out, stream, true,
                     roots, depths);
}

extern "C" fc_status fc_sample_usts_ex(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                                       uint32_t* C, int32_t* parents, uint64_t* visits, uint64_t max_steps_per_tree,
                                       uint64_t* steps_out, void* stream) {
  return sample_impl(g, seed, tau, tree_offset, R, C, parents, visits, max_steps_per_tree, steps_out, stream, true);
}

extern "C" fc_status fc_sample_usts_async(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                                          uint32_t* C, int32_t* parents, uint64_t max_steps_per_tree,
                                          uint64_t* steps_out, void* stream) {
  return sample_impl(g, seed, tau, tree_offset, R, C, parents, nullptr, max_steps_per_tree, steps_out, stream, false);
}

extern "C" fc_status fc_sampler_check(fc_graph* g, void* stream) {
  if (g == nullptr) return fcx::invalid("fc_sampler_check: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t herr = 0;
  FC_CK(cudaMemcpyAsync(&herr, g->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  FC_CK(cudaStreamSynchronize(st));
  FC_CK(cudaMemsetAsync(g->d_err, 0, sizeof(uint32_t), st));
  FC_CK(cudaStreamSynchronize(st));
  if (herr & ERR_OVERFLOW) {
    set_error("fc_sampler_check: a visit counter exceeded 2^24 - 1");
    return FC_EOVERFLOW;
  }
  if (herr & ERR_TIMEOUT) {
    set_error("fc_sampler_check: watchdog iteration budget exhausted");
    return FC_ETIMEOUT;
  }
  if (herr != 0) {
    set_error("fc_sampler_check: internal consistency check failed");
    return FC_ECUDA;
  }
  return FC_OK;
}

namespace {
// device scratch released on the stream when the call returns
struct StreamScratch {
  void* ptr = nullptr;
  cudaStream_t st = nullptr;
  ~StreamScratch() {
    if (ptr) cudaFreeAsync(ptr, st);
  }
};
}  // namespace

static fc_status sample_impl(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R, uint32_t* C,
                             int32_t* parents, uint64_t* visits, uint64_t max_steps_per_tree, uint64_t* steps_out,
                             void* stream, bool sync, int32_t* roots, int32_t* depths) {
  if (g == nullptr || R == nullptr || tau < 0 || tree_offset < 0 || tree_offset + tau > (int64_t(1) << 32) ||
      ((roots != nullptr || depths != nullptr) && !sync)) {
    set_error("fc_sample_usts: bad argument");
    return FC_EINVAL;
  }
  if (tau == 0) return FC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  FC_CK(cudaStreamIsCapturing(st, &cap));
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (capturing && sync) {
    set_error("fc_sample_usts: reads its status back; use fc_sample_usts_async on a capturing stream");
    return FC_EINVAL;
  }
  int dev_smem_optin = 0, nsm = 0;
  FC_CK(cudaDeviceGetAttribute(&dev_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
  FC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device));
  const bool batch = g->num_graphs > 0;
  const int64_t total = (int64_t)(batch ? g->num_graphs : g->n_alpha) * tau;
  const int32_t nmax = batch ? g->max_ng : n;  // largest tree of the launch
  const int wmin = g->walkers > 0 ? g->walkers : 32;
  const bool fits = smem_bytes(wmin, nmax, true) + 64 <= (size_t)dev_smem_optin;
  // automatic placement keeps the state in global memory when the edge-record
  // kernel is requested (it has no shared-memory variant)
  const bool use_smem = g->smem_mode == 2 ? true : (g->smem_mode == 1 ? false : (fits && g->kernel_pref != 2));
  if (use_smem && !fits) {
    set_error("fc_sample_usts: tree state does not fit in shared memory");
    return FC_EINVAL;
  }
  const bool edge = !use_smem && g->edges != nullptr && g->kernel_pref != 1;
  if (g->kernel_pref == 2 && !edge) {
    set_error("fc_sample_usts: the edge-record kernel needs edge records and global tree state");
    return FC_EINVAL;
  }
  // edge-record kernel: CTAs per tree (a thread-block cluster) and where tree
  // membership lives.  Automatic clusters give a launch of few trees enough
  // CTAs to fill the GPU (fc_set_sampler_cluster); the in-tree bitmap goes to
  // shared memory when its share per CTA fits, else membership is a flag in
  // the state words (fc_set_sampler_bitmap; with global tree state forced by
  // the shape, flags); a global-memory bitmap runs without clusters.
  int cl = 1, bits = 0;
  // measured on GB300: popping short cycles from the ring gains 9% on a
  // road-like grid (mean degree 3.7, pops 44% of departures); the prefix
  // buffer stays 6% faster on BA m = 8 (pops 5%)
  const bool ring = edge && (g->pops_mode == 2 || (g->pops_mode == 0 && g->nnz < 8 * (int64_t)g->n));
  // The search queries the occupancy of up to 32 candidate shapes per cluster
  // size (a host cost of milliseconds, which a launch waits for): its results
  // are kept for launches with the same inputs.
  Shape sh;
  const int64_t key[12] = {nmax,      total,     use_smem, edge,        g->bitmap_mode, ring,
                           g->cluster, g->walkers, g->regs, g->weighted, g->root >= 0,  g->smem_mode};
  int hit_slot = -1;
  for (int q = 0; q < fc_graph::SHAPE_SLOTS; ++q)
    if (g->shape_used[q] && std::equal(key, key + 12, g->shape_key[q])) hit_slot = q;
  if (hit_slot >= 0) {
    const int64_t* v = g->shape_val[hit_slot];
    sh.W = (int)v[0];
    sh.regs = (int)v[1];
    sh.per_sm = (int)v[2];
    sh.slots = v[3];
    cl = (int)v[4];
    bits = (int)v[5];
  } else {
    if (edge) {
      const int wmin_e = g->walkers > 0 ? g->walkers : 32;
      auto fits_c = [&](int c) {
        return wilson_edge_smem(wmin_e, nmax, 1, g->weighted, c, ring) + 64 <= (size_t)dev_smem_optin;
      };
      // rooted graphs: state flags, so that several small CTAs share an SM
      auto auto_bits = [&](int c) { return (g->root < 0 && g->smem_mode != 1 && fits_c(c)) ? 1 : 0; };
      int c_util = 1;
      while (c_util < 8 && total * (int64_t)(c_util * 2) <= (int64_t)nsm) c_util *= 2;
      cl = g->cluster > 0 ? g->cluster : c_util;
      if (g->bitmap_mode == 0) {
        bits = auto_bits(cl);
      } else {
        bits = g->bitmap_mode - 1;
        if (bits == 1 && g->cluster == 0)
          while (cl < 8 && !fits_c(cl)) cl *= 2;  // split the bitmap over a larger cluster
        if (bits == 1 && !fits_c(cl)) {
          set_error("fc_sample_usts: the in-tree bitmap does not fit in the shared memory of the cluster");
          return FC_EINVAL;
        }
        if (bits == 2) cl = 1;
      }
      fc_status r = choose_shape(g, nmax, total, use_smem, edge, bits, ring, cl, nsm, dev_smem_optin, &sh);
      if (r != FC_OK) return r;
      // clusters are placed within one GPC, so fewer clusters of 8 are
      // resident than SMs / 8 (15 on GB300's 152 SMs): an automatic cluster
      // is halved until every tree of the launch is in flight at once
      // (measured on GB300, R-MAT n = 2^22, 16 trees: 9.3 ms on clusters of
      // 4 against 18.4 ms in two waves of clusters of 8)
      while (g->cluster == 0 && g->bitmap_mode == 0 && cl > 1 && sh.slots < total) {
        cl /= 2;
        bits = auto_bits(cl);
        sh = Shape();
        r = choose_shape(g, nmax, total, use_smem, edge, bits, ring, cl, nsm, dev_smem_optin, &sh);
        if (r != FC_OK) return r;
      }
    } else {
      const fc_status r = choose_shape(g, nmax, total, use_smem, edge, bits, ring, cl, nsm, dev_smem_optin, &sh);
      if (r != FC_OK) return r;
    }
    const int q = g->shape_next;
    g->shape_next = (q + 1) % fc_graph::SHAPE_SLOTS;
    std::copy(key, key + 12, g->shape_key[q]);
    const int64_t v[6] = {sh.W, sh.regs, sh.per_sm, sh.slots, cl, bits};
    std::copy(v, v + 6, g->shape_val[q]);
    g->shape_used[q] = true;
  }
  const bool sbits = bits == 1;
  const int W = sh.W;
  const size_t shb = edge ? wilson_edge_smem(W, nmax, bits, g->weighted, cl, ring) : smem_bytes(W, nmax, use_smem);
  // trees in flight (each on cl CTAs)
  int64_t grid = std::min<int64_t>(total, std::max<int64_t>(1, sh.slots));
  if (g->max_trees > 0) grid = std::min<int64_t>(grid, g->max_trees);
  void* gstate = nullptr;
  uint32_t* gbits = nullptr;
  unsigned long long* rdpack = nullptr;
  // forest roots and depths: recorded by the edge-record kernel as vertices
  // join the tree (no clusters), else by pointer jumping over the parents
  const bool want_roots = roots != nullptr || depths != nullptr;
  const bool fused_roots = want_roots && edge && cl == 1;
  if (!use_smem) {
    // keep the per-tree state within a quarter of the device memory
    const size_t words = (edge && bits != 2) ? 0 : ((size_t)nmax + 31) / 32;  // global in-tree bitmaps
    const size_t per_tree = (size_t)nmax * sizeof(VState) + ((words * 4 + 255) & ~(size_t)255) +
                            (fused_roots ? (size_t)nmax * 8 : 0);
    const size_t cap_trees = std::max<size_t>(1, (g->device_bytes / 4) / per_tree);
    grid = std::min<int64_t>(grid, (int64_t)cap_trees);
    void* ws = nullptr;  // state (and global bitmaps) of `grid` tree slots
    const fc_status s = sampler_scratch(g->device, (size_t)grid * per_tree, st, &ws, capturing);
    if (s != FC_OK) return s;
    gstate = ws;
    gbits = (uint32_t*)((char*)ws + (size_t)grid * nmax * sizeof(VState));
    if (fused_roots)
      rdpack = (unsigned long long*)((char*)ws + (size_t)grid * nmax * sizeof(VState) +
                                     (size_t)grid * ((words * 4 + 255) & ~(size_t)255));
  }
  g->last_W = W;
  g->last_regs = sh.regs;
  g->last_grid = (int32_t)(grid * cl);
  g->last_kernel = edge ? 2 + bits : 1;
  g->last_cluster = cl;
  WParams p;
  p.n = n;
  p.n_alpha = g->n_alpha;
  p.nnz = g->nnz;
  p.rowinfo = g->rowinfo;
  p.colidx = g->colidx;
  p.order = g->order;
  p.B = g->weighted ? g->B : nullptr;
  p.tau = tau;
  p.tree_offset = tree_offset;
  // automatic start order: vertex id (start windows load coalesced), except
  // when the numbering follows the geometry (neighbouring starts would collide)
  p.descending = g->order_auto ? 0 : g->order_desc;
  p.id_order = g->order_auto ? !g->id_local : g->order_id;

  p.edges = g->edges;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  p.R = R;
  p.C = C;
  p.parents = parents;
  const size_t prow = (size_t)(batch ? tau : (int64_t)g->n_alpha * tau);  // parent rows of the call
  StreamScratch pscr;
  pscr.st = st;
  p.roots = fused_roots ? roots : nullptr;
  p.depths = fused_roots ? depths : nullptr;
  p.rdpack = rdpack;
  if (want_roots && !fused_roots && parents == nullptr) {  // pointer jumping needs the parents
    FC_CK(cudaMallocAsync(&pscr.ptr, prow * (size_t)n * sizeof(int32_t), st));
    p.parents = (int32_t*)pscr.ptr;
  }
  p.visits = (unsigned long long*)visits;
  p.steps = steps_out;
  p.gstate = (VState*)gstate;
  p.gbits = gbits;
  p.words = (int32_t)(((int64_t)nmax + 31) / 32);
  p.nmax = nmax;
  p.num_graphs = g->num_graphs;
  p.voff = g->voff;
  p.gorder = g->gorder;
  p.item_ns = nullptr;
  p.t0_ns = nullptr;
  // walks on G with one exit: warp w of a CTA starts walks once its tree
  // holds w n / 256 vertices.  Measured on GB300 (BA n = 2^20 rooted at its
  // hub, 1024 trees, 128 walkers per tree): iterations in conflict waits 0.73
  // -> 0.15 per departure, repeated departures 9% -> 0.5%, sampling 246 ->
  // 211 ms.  A tree's growth stays sequential while it is small (a walk
  // needs about 2m / vol(tree) steps to hit it), so larger shapes (1024
  // walkers, in-tree bitmap) with the ramp ran no faster (214 ms).
  p.ramp_q = (edge && cl == 1 && g->root >= 0) ? (uint32_t)std::max<int64_t>(1, (int64_t)nmax >> 8) : 0u;
  if (batch) {
    const size_t items = (size_t)g->num_graphs * (size_t)tau;
    if (g->item_cap < items && capturing) {
      set_error("fc_sample_usts_async: batch timestamps must be sized by an uncaptured call before stream capture");
      return FC_EINVAL;
    }
    if (g->item_cap < items) {
      if (g->item_ns) FC_CK(cudaFreeAsync(g->item_ns, st));
      FC_CK(cudaMallocAsync((void**)&g->item_ns, items * sizeof(unsigned long long), st));
      g->item_cap = items;
    }
    g->last_tau = tau;
    p.item_ns = g->item_ns;
    p.t0_ns = g->t0_ns;
    FC_CK(cudaMemsetAsync(g->t0_ns, 0xff, sizeof(unsigned long long), st));
  }
  p.counter = g->d_counter;
  p.err = g->d_err;
  p.stats = g->d_stats;
  {
    // default watchdog: 8 n + 2^20 iterations per walker on G* (every step can
    // exit to u*); walks on G with one exit (fc_build_rooted) take
    // sum_v d_w(v) r(root, v) steps in all, up to quadratic in n on long
    // paths, and walkers wait for each other longer: 2^26 + 64 n
    const uint64_t mi = max_steps_per_tree ? max_steps_per_tree
                        : (g->root >= 0 ? (1ull << 26) + (uint64_t)64 * (uint64_t)n
                                        : (uint64_t)8 * (uint64_t)n + (1ull << 20));
    p.max_iters = (uint32_t)std::min<uint64_t>(mi, 0xffffffffull);
  }
  p.pre_cleared = 0;
  if (!use_smem) {
    // clear the state and bitmaps of the first wave in one pass
    const size_t words = (edge && bits != 2) ? 0 : ((size_t)nmax + 31) / 32;
    FC_CK(cudaMemsetAsync(gstate, 0, (size_t)grid * nmax * sizeof(VState) + (size_t)grid * words * 4, st));
    p.pre_cleared = 1;
  }
  FC_CK(cudaMemsetAsync(g->d_counter, 0, sizeof(unsigned long long), st));
  if (sync) FC_CK(cudaMemsetAsync(g->d_err, 0, sizeof(uint32_t), st));
  FC_CK(cudaMemsetAsync(g->d_stats, 0, (2 + N_CNT) * sizeof(unsigned long long), st));
  const WilsonFn fn = edge ? wilson_edge_fn(bits, g->weighted, ring, cl > 1, sh.regs, fused_roots)
                            : wilson_fn(use_smem, sh.regs);
  if (use_smem || edge) FC_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
  if (cl > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid * cl));
    cfg.blockDim = dim3((unsigned)W);
    cfg.dynamicSmemBytes = shb;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int resident = 0;
    FC_CK(cudaOccupancyMaxActiveClusters(&resident, fn, &cfg));
    if (resident < 1) {
      set_error("fc_sample_usts: a cluster of this size and shape cannot be resident");
      return FC_EINVAL;
    }
    FC_CK(cudaLaunchKernelEx(&cfg, fn, p));
  } else {
    fn<<<(unsigned)grid, W, shb, st>>>(p);
  }
  FC_LAUNCHED();
  if (!sync) return FC_OK;
  uint32_t herr = 0;
  FC_CK(cudaMemcpyAsync(&herr, g->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  FC_CK(cudaStreamSynchronize(st));
  if (herr & ERR_OVERFLOW) {
    set_error("fc_sample_usts: a visit counter exceeded 2^24 - 1");
    return FC_EOVERFLOW;
  }
  if (herr & ERR_TIMEOUT) {
    set_error("fc_sample_usts: watchdog iteration budget exhausted");
    return FC_ETIMEOUT;
  }
  if (herr != 0) {
    set_error("fc_sample_usts: internal consistency check failed");
    return FC_ECUDA;
  }
  if (want_roots && !fused_roots) {
    StreamScratch r2;
    r2.st = st;
    if (roots == nullptr) FC_CK(cudaMallocAsync(&r2.ptr, prow * (size_t)n * sizeof(int32_t), st));
    const fc_status s = fc_tree_roots(p.parents, n, (int64_t)prow, roots ? roots : (int32_t*)r2.ptr, depths, st);
    if (s != FC_OK) return s;
  }
  return FC_OK;
}

// Work counters of the last fc_sample_usts call on g: stack pops (summed over
// trees) and departures (walk steps actually executed, including steps redone
// after a released path).  Host pointers; either may be NULL.  Synchronous.
extern "C" fc_status fc_sampler_stats(fc_graph* g, uint64_t* pops, uint64_t* departures) {
  if (g == nullptr) return fcx::invalid("fc_sampler_stats: bad argument");
  unsigned long long h[2] = {0, 0};
  FC_CK(cudaMemcpy(h, g->d_stats, sizeof(h), cudaMemcpyDeviceToHost));
  if (pops) *pops = h[0];
  if (departures) *departures = h[1];
  return FC_OK;
}

extern "C" fc_status fc_sampler_counters(fc_graph* g, uint64_t* out, int32_t count) {
  if (g == nullptr || out == nullptr || count < 0) return fcx::invalid("fc_sampler_counters: bad argument");
  unsigned long long h[N_CNT] = {};
  FC_CK(cudaMemcpy(h, g->d_stats + 2, sizeof(h), cudaMemcpyDeviceToHost));
  for (int i = 0; i < count && i < N_CNT; ++i) out[i] = h[i];
  return N_CNT <= count ? FC_OK : FC_EINVAL;
}

extern "C" fc_status fc_stack_entries(fc_graph* g, int32_t alpha_idx, uint64_t seed, uint32_t tree, int64_t count,
                                      const int32_t* verts, const uint32_t* ks, int32_t* out, void* stream) {
  if (g == nullptr || alpha_idx < 0 || alpha_idx >= g->n_alpha || count < 0 ||
      (count > 0 && (verts == nullptr || ks == nullptr || out == nullptr))) {
    set_error("fc_stack_entries: bad argument");
    return FC_EINVAL;
  }
  if (count == 0) return FC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  WParams p = {};
  p.n = g->n;
  p.n_alpha = g->n_alpha;
  p.nnz = g->nnz;
  p.rowinfo = g->rowinfo;
  p.colidx = g->colidx;
  p.B = g->weighted ? g->B : nullptr;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  p.err = g->d_err;
  k_stack_entries<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(p, alpha_idx, tree, count, verts, ks, out);
  FC_LAUNCHED();
  return FC_OK;
}

extern "C" fc_status fc_batch_latency(fc_graph* g, double* per_graph_ms) {
  if (g == nullptr || per_graph_ms == nullptr || g->num_graphs < 1 || g->item_ns == nullptr || g->last_tau < 1) {
    set_error("fc_batch_latency: no batch launch recorded");
    return FC_EINVAL;
  }
  const size_t items = (size_t)g->num_graphs * (size_t)g->last_tau;
  std::vector<unsigned long long> h(items);
  unsigned long long t0 = 0;
  FC_CK(cudaMemcpy(h.data(), g->item_ns, items * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  FC_CK(cudaMemcpy(&t0, g->t0_ns, sizeof(t0), cudaMemcpyDeviceToHost));
  for (int32_t gi = 0; gi < g->num_graphs; ++gi) {
    unsigned long long mx = 0;
    for (int64_t t = 0; t < g->last_tau; ++t) mx = std::max(mx, h[(size_t)gi * g->last_tau + t]);
    per_graph_ms[gi] = mx > t0 ? (double)(mx - t0) * 1e-6 : 0.0;
  }
  return FC_OK;
}
