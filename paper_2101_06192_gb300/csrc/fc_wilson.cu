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
  const uint4* rowinfo;     // [n_alpha][n]
  const int32_t* colidx;    // [nnz]
  const uint64_t* B;        // [n_alpha][nnz] or null (unweighted)
  const int32_t* order;     // [n]
  int64_t tau;
  int64_t tree_offset;
  uint32_t key0, key1;
  uint32_t* R;              // [n_alpha][n]
  uint32_t* C;              // [n_alpha][n] or null
  int32_t* parents;         // [n_alpha*tau][n] or null
  uint64_t* steps;          // [n_alpha*tau] or null
  VState* gstate;           // [gridDim.x][n] (global-state variant)
  unsigned long long* counter;
  uint32_t* err;
  unsigned long long* stats;  // [0] pops, [1] departures
  uint64_t max_iters;
};

// Vertex selected by the stack entry with Philox words o at a vertex with row
// info ri = {row offset, degree, T lo, T hi}.  n means u*.
__device__ __forceinline__ uint32_t select_vertex(const WParams& p, const uint4& ri, const uint4& o,
                                                  const uint64_t* __restrict__ Brow) {
  const uint64_t u = stack_u53(o);
  const uint64_t T = (uint64_t)ri.z | ((uint64_t)ri.w << 32);
  if (u < T) return (uint32_t)p.n;
  if (Brow == nullptr) {
    const uint32_t j = __umulhi(o.z, ri.y);  // floor(o2 d / 2^32)
    return (uint32_t)__ldg(p.colidx + ri.x + j);
  }
  // first entry j of the row with u < B[j]; the last entry is 2^53 > u
  uint32_t lo = 0, hi = ri.y - 1;
  const uint64_t* b = Brow + ri.x;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (u < __ldg(b + mid)) hi = mid; else lo = mid + 1;
  }
  return (uint32_t)__ldg(p.colidx + ri.x + lo);
}

enum { M_IDLE = 0, M_CLAIM = 1, M_WAIT = 2 };

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* a) {
  return *(const volatile unsigned long long*)a;
}

template <bool SMEM>
__global__ void __launch_bounds__(1024) k_wilson(WParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long sh_tree, sh_pops, sh_deps;
  __shared__ uint32_t sh_next;
  __shared__ volatile uint32_t sh_abort;
  const int me = threadIdx.x;
  const int W = blockDim.x;
  const int lane = me & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  volatile uint32_t* sh_gen = (volatile uint32_t*)smem_raw;
  VState* S;
  if (SMEM) {
    S = (VState*)(smem_raw + (((size_t)W * 4 + 15) & ~(size_t)15));
  } else {
    S = p.gstate + (size_t)blockIdx.x * p.n;
  }
  const int32_t n = p.n;
  const int64_t total = (int64_t)p.n_alpha * p.tau;

  for (;;) {
    if (me == 0) sh_tree = atomicAdd(p.counter, 1ull);
    __syncthreads();
    const unsigned long long tree = sh_tree;
    if ((int64_t)tree >= total || *(volatile uint32_t*)p.err != 0u) break;
    const int a = (int)(tree / (unsigned long long)p.tau);
    const uint32_t tg = (uint32_t)(p.tree_offset + (int64_t)(tree % (unsigned long long)p.tau));
    for (int32_t v = me; v < n; v += W) reinterpret_cast<uint4*>(S)[v] = make_uint4(0u, 0u, 0u, 0u);
    sh_gen[me] = 1u;
    if (me == 0) {
      sh_next = 0;
      sh_abort = 0;
      sh_pops = 0;
      sh_deps = 0;
    }
    __syncthreads();

    const uint4* __restrict__ rinfo = p.rowinfo + (size_t)a * n;
    const uint64_t* Brow = p.B ? p.B + (size_t)a * p.nnz : nullptr;
    uint32_t* Ra = p.R + (size_t)a * n;
    uint32_t* Ca = p.C ? p.C + (size_t)a * n : nullptr;

    int mode = M_IDLE;
    bool done = false;
    int32_t s = 0, x = 0, h = -1;
    uint32_t gen = 1;
    unsigned long long wait_tag = 0, confirm_tag = 0;
    uint64_t iters = 0;
    unsigned long long pops = 0, deps = 0;

    while (true) {
      __syncwarp();
      const bool stop = done || (sh_abort != 0u);
      if (__all_sync(FULL, stop)) break;
      // hand consecutive start indices (ascending degree) to the idle lanes
      const unsigned need = __ballot_sync(FULL, !stop && mode == M_IDLE);
      if (need) {
        const int leader = __ffs(need) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&sh_next, (uint32_t)__popc(need));
        base = __shfl_sync(FULL, base, leader);
        if (!stop && mode == M_IDLE) {
          const uint32_t i = base + __popc(need & lt_mask);
          if (i >= (uint32_t)n) {
            done = true;
          } else {
            s = __ldg(p.order + i);
            x = s;
            h = -1;
            mode = M_CLAIM;
            confirm_tag = 0;
          }
        }
      }
      if (stop || done) continue;
      if (++iters > p.max_iters) {
        atomicOr(p.err, ERR_TIMEOUT);
        sh_abort = 1u;
        done = true;
        continue;
      }

      if (mode == M_WAIT) {
        // holding nothing: wait until x leaves the path it was blocked by
        const unsigned long long cur = ld_volatile(&S[x].st) >> K_BITS;
        const uint32_t ww = (uint32_t)(wait_tag & ((1u << W_BITS) - 1));
        if (cur == wait_tag && sh_gen[ww] == (uint32_t)(wait_tag >> W_BITS)) continue;
        mode = M_CLAIM;
        x = s;
        h = -1;
        confirm_tag = 0;
      }

      // ---- try to take x onto this walker's path ----
      const uint4 ri = __ldg(rinfo + x);
      const unsigned long long mytag = ((unsigned long long)gen << W_BITS) | (unsigned)me;
      const unsigned long long old = atomicCAS(&S[x].st, 0ull, mytag << K_BITS);
      uint4 o = philox4x32_10(0u, (uint32_t)x, tg, (uint32_t)a, p.key0, p.key1);
      uint32_t k = 0;
      if (old != 0ull) {
        const unsigned long long tag = old >> K_BITS;
        if (tag == 0ull) {
          // free vertex whose stack has been popped before
          const unsigned long long want = (mytag << K_BITS) | (old & K_MASK);
          if (atomicCAS(&S[x].st, old, want) != old) continue;  // raced: retry
          k = (uint32_t)(old & K_MASK);
          if (k >= (uint32_t)K_MASK) {
            atomicOr(p.err, ERR_OVERFLOW);
            sh_abort = 1u;
            done = true;
            continue;
          }
          o = philox4x32_10(k, (uint32_t)x, tg, (uint32_t)a, p.key0, p.key1);
        } else {
          const uint32_t w = (uint32_t)(tag & ((1u << W_BITS) - 1));
          const uint32_t tgen = (uint32_t)(tag >> W_BITS);
          bool in_tree = false;
          if (w == (uint32_t)me) {
            if (tgen == gen) {
              // x is on this walker's own path: pop the cycle x -> ... -> h -> x
              uint32_t v = S[x].nxt;
              int32_t guard = 0;
              while (v != (uint32_t)x && guard++ <= n) {
                const uint32_t nv = S[v].nxt;
                atomicAdd(&S[v].st, 1ull - (mytag << K_BITS));  // free, next entry
                ++pops;
                v = nv;
              }
              k = (uint32_t)(old & K_MASK) + 1u;
              if (k >= (uint32_t)K_MASK || v != (uint32_t)x) {
                atomicOr(p.err, k >= (uint32_t)K_MASK ? ERR_OVERFLOW : ERR_INVAL);
                sh_abort = 1u;
                done = true;
                continue;
              }
              atomicAdd(&S[x].st, 1ull);
              ++pops;
              o = philox4x32_10(k, (uint32_t)x, tg, (uint32_t)a, p.key0, p.key1);
            } else {
              in_tree = true;  // a finished path of this walker
            }
          } else {
            const uint32_t gcur = sh_gen[w];
            if (gcur == tgen) {
              // x is on walker w's active path
              confirm_tag = 0;
              if (h < 0 || (uint32_t)me < w) continue;  // wait (retry next iteration)
              // die: give the whole path back, stacks untouched
              uint32_t v = (uint32_t)s;
              int32_t guard = 0;
              while (guard++ <= n) {
                const uint32_t nv = S[v].nxt;
                atomicAdd(&S[v].st, 0ull - (mytag << K_BITS));
                if (v == (uint32_t)h) break;
                v = nv;
              }
              h = -1;
              mode = M_WAIT;
              wait_tag = tag;
              continue;
            }
            // w has finished generation tgen; confirm with a second read of x
            // ordered after the generation read (x may have been popped from
            // w's path between our CAS and that read)
            if (confirm_tag != tag) {
              confirm_tag = tag;
              __threadfence_block();
              continue;
            }
            in_tree = true;
          }
          if (in_tree) {
            // the path s -> ... -> h reaches the tree through x
            if (h >= 0) {
              __threadfence_block();
              ++gen;
              sh_gen[me] = gen;
            }
            h = -1;
            mode = M_IDLE;
            confirm_tag = 0;
            continue;
          }
        }
      }
      // ---- x is the new head, at stack entry k ----
      confirm_tag = 0;
      h = x;
      const uint32_t t = select_vertex(p, ri, o, Brow);
      S[h].nxt = t;
      ++deps;
      if (t == (uint32_t)n) {
        // the loop-erased walk ends with the edge {h, u*} (Algorithm 2: R[h]++)
        atomicAdd(Ra + h, 1u);
        if (Ca != nullptr && k == 0u) atomicAdd(Ca + h, 1u);
        __threadfence_block();
        ++gen;
        sh_gen[me] = gen;
        h = -1;
        mode = M_IDLE;
        continue;
      }
      x = (int32_t)t;
    }

    atomicAdd(&sh_pops, pops);
    atomicAdd(&sh_deps, deps);
    __syncthreads();
    if (p.parents != nullptr) {
      int32_t* par = p.parents + (size_t)tree * n;
      for (int32_t v = me; v < n; v += W) par[v] = (int32_t)S[v].nxt;
    }
    if (me == 0) {
      if (p.steps != nullptr) p.steps[tree] = (uint64_t)n + sh_pops;
      atomicAdd(&p.stats[0], sh_pops);
      atomicAdd(&p.stats[1], sh_deps);
    }
    __syncthreads();
  }
}

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
  out[i] = (int32_t)select_vertex(p, ri, o, p.B ? p.B + (size_t)a * p.nnz : nullptr);
}

static size_t smem_bytes(int W, int32_t n, bool smem) {
  const size_t gen = ((size_t)W * 4 + 15) & ~(size_t)15;
  return smem ? gen + (size_t)n * sizeof(VState) : gen;
}

static int default_walkers(int32_t n) {
  int w = (n / 64) & ~31;
  return std::max(32, std::min(256, w));
}

}  // namespace fcx

using namespace fcx;

extern "C" fc_status fc_sample_usts(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                                    uint32_t* C, int32_t* parents, uint64_t max_steps_per_tree,
                                    uint64_t* steps_out, void* stream) {
  if (g == nullptr || R == nullptr || tau < 0 || tree_offset < 0 || tree_offset + tau > (int64_t(1) << 32)) {
    set_error("fc_sample_usts: bad argument");
    return FC_EINVAL;
  }
  if (tau == 0) return FC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  const int W = g->walkers > 0 ? g->walkers : default_walkers(n);
  int dev_smem_optin = 0, nsm = 0;
  FC_CK(cudaDeviceGetAttribute(&dev_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
  FC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device));
  const bool fits = smem_bytes(W, n, true) + 64 <= (size_t)dev_smem_optin;
  bool use_smem = g->smem_mode == 2 ? true : (g->smem_mode == 1 ? false : fits);
  if (use_smem && !fits) {
    set_error("fc_sample_usts: tree state does not fit in shared memory");
    return FC_EINVAL;
  }
  const size_t shb = smem_bytes(W, n, use_smem);
  int per_sm = 0;
  if (use_smem) {
    FC_CK(cudaFuncSetAttribute(k_wilson<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
    FC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wilson<true>, W, shb));
  } else {
    FC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wilson<false>, W, shb));
  }
  if (per_sm < 1) {
    set_error("fc_sample_usts: launch shape does not fit on an SM");
    return FC_EINVAL;
  }
  const int64_t total = (int64_t)g->n_alpha * tau;
  int64_t grid = std::min<int64_t>(total, (int64_t)per_sm * nsm);
  if (g->max_trees > 0) grid = std::min<int64_t>(grid, g->max_trees);
  void* gstate = nullptr;
  if (!use_smem) {
    // keep the per-tree state within a quarter of the device memory
    size_t freeb = 0, totalb = 0;
    FC_CK(cudaMemGetInfo(&freeb, &totalb));
    const size_t per_tree = (size_t)n * sizeof(VState);
    const size_t cap_trees = std::max<size_t>(1, (totalb / 4) / per_tree);
    grid = std::min<int64_t>(grid, (int64_t)cap_trees);
    void* ws = nullptr;
    const fc_status s = sampler_scratch(g->device, (size_t)grid * per_tree, st, &ws);
    if (s != FC_OK) return s;
    g->ws = nullptr;
    gstate = ws;
  }
  WParams p;
  p.n = n;
  p.n_alpha = g->n_alpha;
  p.nnz = g->nnz;
  p.rowinfo = g->rowinfo;
  p.colidx = g->colidx;
  p.B = g->weighted ? g->B : nullptr;
  p.order = g->order;
  p.tau = tau;
  p.tree_offset = tree_offset;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  p.R = R;
  p.C = C;
  p.parents = parents;
  p.steps = steps_out;
  p.gstate = (VState*)gstate;
  p.counter = g->d_counter;
  p.err = g->d_err;
  p.stats = g->d_stats;
  p.max_iters = max_steps_per_tree ? max_steps_per_tree : (uint64_t)8 * (uint64_t)n + (1ull << 20);
  FC_CK(cudaMemsetAsync(g->d_counter, 0, sizeof(unsigned long long), st));
  FC_CK(cudaMemsetAsync(g->d_err, 0, sizeof(uint32_t), st));
  FC_CK(cudaMemsetAsync(g->d_stats, 0, 2 * sizeof(unsigned long long), st));
  if (use_smem)
    k_wilson<true><<<(unsigned)grid, W, shb, st>>>(p);
  else
    k_wilson<false><<<(unsigned)grid, W, shb, st>>>(p);
  FC_LAUNCHED();
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
  return FC_OK;
}

// Work counters of the last fc_sample_usts call on g: stack pops (summed over
// trees) and departures (walk steps actually executed, including steps redone
// after a released path).  Host pointers; either may be NULL.  Synchronous.
extern "C" fc_status fc_sampler_stats(fc_graph* g, uint64_t* pops, uint64_t* departures) {
  if (g == nullptr) return FC_EINVAL;
  unsigned long long h[2] = {0, 0};
  FC_CK(cudaMemcpy(h, g->d_stats, sizeof(h), cudaMemcpyDeviceToHost));
  if (pops) *pops = h[0];
  if (departures) *departures = h[1];
  return FC_OK;
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
