// G* builder (Sec. 4.1; first step of Algorithm 1): CSR validation, degrees,
// FP64 weight prefixes, ascending-degree start order (Algorithm 2) and the
// integer thresholds of the random-stack selector.  Also the shared error
// plumbing and the small graph-management entry points of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <atomic>
#include <mutex>

#include "fc_internal.cuh"

namespace fcx {

// Record msg as the last error and return FC_EINVAL.
static inline fc_status invalid(const char* msg) {
  set_error(msg);
  return FC_EINVAL;
}

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};
static std::mutex g_scratch_mu;
static Scratch g_scratch[64];

fc_status sampler_scratch(int device, size_t bytes, cudaStream_t st, void** out, bool capturing) {
  if (device < 0 || device >= 64) return FC_EINVAL;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  Scratch& sc = g_scratch[device];
  if (sc.bytes < bytes && capturing) {
    set_error("fc_sample_usts_async: sampler scratch must be sized by an uncaptured call before stream capture");
    return FC_EINVAL;
  }
  if (sc.bytes < bytes) {
    if (sc.ptr) {
      FC_CK(cudaDeviceSynchronize());
      FC_CK(cudaFree(sc.ptr));
      sc.ptr = nullptr;
      sc.bytes = 0;
    }
    FC_CK(cudaMalloc(&sc.ptr, bytes));
    sc.bytes = bytes;
  }
  (void)st;
  *out = sc.ptr;
  return FC_OK;
}

static bool g_pool_set[64] = {};
void retain_pool(int device) {
  if (device < 0 || device >= 64 || g_pool_set[device]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  g_pool_set[device] = true;
}

fc_status cuda_fail(cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? FC_ENOMEM : FC_ECUDA;
}

// ---------------------------------------------------------------------------
// Validation: one warp per row.  Every index is bounds-checked before use, so
// a malformed CSR sets the error word instead of touching memory out of range.
// ---------------------------------------------------------------------------
__global__ void k_validate(int32_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ colidx, const float* __restrict__ w,
                           const int32_t* __restrict__ gid, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int64_t b = rowptr[v], e = rowptr[v + 1];
    bool bad = false;
    if (v == 0 && b != 0) bad = true;
    if (v == n - 1 && e != nnz) bad = true;
    if (b < 0 || e < b || e > nnz) bad = true;
    if (bad) {
      if (lane == 0) atomicOr(err, ERR_INVAL);
      continue;
    }
    for (int64_t i = b + lane; i < e; i += 32) {
      const int32_t c = colidx[i];
      bool ok = c >= 0 && c < n && c != v;
      if (ok && gid != nullptr && gid[c] != gid[v]) ok = false;  // batch: edges stay in their graph
      if (ok && i > b && colidx[i - 1] >= c) ok = false;  // sorted, no duplicates
      float wv = 1.0f;
      if (ok && w != nullptr) {
        wv = w[i];
        if (!(isfinite(wv) && wv >= 0.0f)) ok = false;
      }
      if (ok) {  // symmetric: v must appear in row c with the same weight
        int64_t lo = rowptr[c], hi = rowptr[c + 1];
        if (lo < 0) lo = 0;
        if (hi > nnz) hi = nnz;
        bool found = false;
        for (int it = 0; it < 64 && lo < hi; ++it) {
          const int64_t mid = lo + (hi - lo) / 2;
          const int32_t cm = colidx[mid];
          if (cm == v) {
            found = (w == nullptr) || (w[mid] == wv);
            break;
          }
          if (cm < v) lo = mid + 1; else hi = mid;
        }
        ok = found;
      }
      if (!ok) atomicOr(err, ERR_INVAL);
    }
  }
}

// Degrees, weighted degrees and the per-row prefix of the weights, summed left
// to right in FP64 (one thread per row keeps the summation order fixed).
__global__ void k_degrees(int32_t n, const int64_t* __restrict__ rowptr, const float* __restrict__ w,
                          int32_t* __restrict__ deg, double* __restrict__ dw, double* __restrict__ S,
                          int32_t* max_deg) {
  int32_t local_max = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rowptr[v], e = rowptr[v + 1];
    const int32_t d = (int32_t)(e - b);
    deg[v] = d;
    if (w != nullptr) {
      double s = 0.0;
      for (int64_t i = b; i < e; ++i) {
        s = __dadd_rn(s, (double)w[i]);
        S[i] = s;
      }
      dw[v] = s;
    } else {
      dw[v] = (double)d;
    }
    local_max = max(local_max, d);
  }
  local_max = __reduce_max_sync(0xffffffffu, local_max);
  if ((threadIdx.x & 31) == 0 && local_max > 0) atomicMax(max_deg, local_max);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (degree, vertex) by degree, 8-bit digits.  One warp
// per tile of 1024 items, processed as 32 consecutive chunks so that equal
// digits keep their input (= vertex id) order.
// ---------------------------------------------------------------------------
constexpr int RS_TILE = 1024;

__global__ void k_rs_hist(int32_t n, const uint32_t* __restrict__ keys, int shift,
                          uint32_t* __restrict__ hist, int32_t nblk) {
  __shared__ uint32_t cnt[256];
  const int lane = threadIdx.x;
  for (int d = lane; d < 256; d += 32) cnt[d] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int c = 0; c < RS_TILE / 32; ++c) {
    const int64_t i = base + c * 32 + lane;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
  }
  __syncwarp();
  for (int d = lane; d < 256; d += 32) hist[(int64_t)d * nblk + blockIdx.x] = cnt[d];
}

__global__ void k_rs_scatter(int32_t n, const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int shift,
                             const uint32_t* __restrict__ offs, int32_t nblk) {
  __shared__ uint32_t run[256];
  const int lane = threadIdx.x;
  for (int d = lane; d < 256; d += 32) run[d] = offs[(int64_t)d * nblk + blockIdx.x];
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < RS_TILE / 32; ++c) {
    const int64_t i = base + c * 32 + lane;
    const bool valid = i < n;
    uint32_t key = 0;
    int32_t val = 0;
    uint32_t d = 256u + lane;  // unique dummy digit for padding lanes
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = (key >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt);
    if (valid) {
      const uint32_t pos = run[d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) run[d] += __popc(peers);
    __syncwarp();
  }
}

// Exclusive scan of uint32 (block of 1024 threads per 1024 items).
__global__ void k_scan_block(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t len,
                             uint32_t* __restrict__ sums) {
  __shared__ uint32_t wsum[32];
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  const uint32_t x = i < len ? in[i] : 0u;
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
    uint32_t t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  const uint32_t incl = s + (wid > 0 ? wsum[wid - 1] : 0u);
  if (i < len) out[i] = incl - x;
  if (threadIdx.x == 1023 && sums != nullptr) sums[blockIdx.x] = incl;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t len, const uint32_t* __restrict__ add) {
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  if (i < len) out[i] += add[blockIdx.x];
}

fc_status exclusive_scan(const uint32_t* in, uint32_t* out, int64_t len, cudaStream_t st) {
  const int64_t nb = (len + 1023) / 1024;
  if (nb <= 1) {
    k_scan_block<<<1, 1024, 0, st>>>(in, out, len, nullptr);
    FC_LAUNCHED();
    return FC_OK;
  }
  uint32_t *sums = nullptr, *sums_x = nullptr;
  FC_CK(cudaMallocAsync((void**)&sums, nb * sizeof(uint32_t), st));
  FC_CK(cudaMallocAsync((void**)&sums_x, nb * sizeof(uint32_t), st));
  k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(in, out, len, sums);
  FC_LAUNCHED();
  fc_status r = exclusive_scan(sums, sums_x, nb, st);
  if (r == FC_OK) {
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, len, sums_x);
    FC_LAUNCHED();
  }
  FC_CK(cudaFreeAsync(sums, st));
  FC_CK(cudaFreeAsync(sums_x, st));
  return r;
}

__global__ void k_iota_keys(int32_t n, const int32_t* __restrict__ deg, uint32_t* __restrict__ keys,
                            int32_t* __restrict__ vals) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    keys[v] = (uint32_t)deg[v];
    vals[v] = (int32_t)v;
  }
}

// ---------------------------------------------------------------------------
// Selector thresholds for one alpha.
//   T_v = count_below(gamma, t_v): stack entries selecting u* (slot 0),
//   B_e = count_below(t_j, t_v) for the entry e of slot j (weighted rows),
// with t_v = fl(gamma + fl(alpha s_v)), s_v = d_v (unweighted) or d_w(v)
// (weighted), t_j = fl(gamma + fl(alpha S_j)).  gamma = 1 on G* (the edge to
// u*).  Walks on G rooted at a vertex (fc_build_rooted) take gamma = 0 and
// alpha = 1 (no exit to u*, neighbours in proportion to w), except at the
// root, whose every stack entry selects u* (T = 2^53): the sampled tree of
// G* is then {root, u*} plus a uniform spanning tree of G rooted at the root.
// ---------------------------------------------------------------------------
__global__ void k_thr_vertex(int32_t n, double alpha_s, const double* __restrict__ alpha_v, bool weighted,
                             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ deg,
                             const double* __restrict__ dw, double gamma, int32_t root,
                             uint4* __restrict__ rowinfo) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const double alpha = alpha_v ? alpha_v[v] : alpha_s;
    const int32_t d = deg[v];
    const double t = deg_gamma(gamma, alpha, weighted ? dw[v] : (double)d);
    const uint64_t T = v == root ? TWO53 : count_below(gamma, t);
    rowinfo[v] = make_uint4((uint32_t)rowptr[v], (uint32_t)d, (uint32_t)T, (uint32_t)(T >> 32));
  }
}

__global__ void k_thr_nnz(int32_t n, double alpha_s, const double* __restrict__ alpha_v,
                          const int64_t* __restrict__ rowptr, const double* __restrict__ S,
                          const double* __restrict__ dw, double gamma, uint64_t* __restrict__ B) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const double alpha = alpha_v ? alpha_v[v] : alpha_s;
    const double t = deg_gamma(gamma, alpha, dw[v]);
    for (int64_t e = rowptr[v] + lane; e < rowptr[v + 1]; e += 32)
      B[e] = count_below(deg_gamma(gamma, alpha, S[e]), t);
  }
}

// graph of each vertex (binary search over the vertex offsets) and its alpha
__global__ void k_batch_vertex(int32_t n, int32_t G, const int64_t* __restrict__ voff,
                               const double* __restrict__ galpha, int32_t* __restrict__ gid,
                               double* __restrict__ alpha_v, uint32_t* __restrict__ keys) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = G - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (voff[mid] <= v) lo = mid; else hi = mid - 1;
    }
    gid[v] = lo;
    alpha_v[v] = galpha[lo];
  }
  (void)keys;
}

// keys[i] = graph of order[i] (second, stable sort pass of the batch start order)
__global__ void k_gid_keys(int32_t n, const int32_t* __restrict__ order, const int32_t* __restrict__ gid,
                           uint32_t* __restrict__ keys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = (uint32_t)gid[order[i]];
}

static int grid_for(int64_t items, int threads) {
  int64_t b = (items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (int)b;
}

// Locality of the vertex numbering: CSR entries whose endpoints are at most 32
// ids apart (high for meshes and road networks numbered along their geometry).
// Each thread takes a run of 64 entries (its first row by binary search), so
// the entries are read in order whatever the degrees.
constexpr int LOC_RUN = 64;
__global__ void k_id_locality(int32_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colidx, unsigned long long* count) {
  unsigned long long local = 0;
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * LOC_RUN;
  if (e0 < nnz) {
    const int64_t e1 = e0 + LOC_RUN < nnz ? e0 + LOC_RUN : nnz;
    int32_t lo = 0, hi = n - 1;  // the row v with rowptr[v] <= e0 < rowptr[v + 1]
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo + 1) / 2;
      if (rowptr[mid] <= e0) lo = mid;
      else hi = mid - 1;
    }
    int64_t v = lo, end = rowptr[v + 1];
    for (int64_t e = e0; e < e1; ++e) {
      while (e >= end) end = rowptr[++v + 1];
      const int64_t d = (int64_t)colidx[e] - v;
      local += (d >= -32 && d <= 32) ? 1ull : 0ull;
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// Edge records of the edge-record sampler: for CSR entry e with target t,
// {t, row offset of t, degree of t, min(T_t >> 21, 2^32 - 1)}.
__global__ void k_edge_records(int64_t nnz, const int32_t* __restrict__ colidx, const uint4* __restrict__ rowinfo,
                               uint4* __restrict__ edges) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = colidx[e];
    const uint4 ri = rowinfo[t];
    const uint64_t T = (uint64_t)ri.z | ((uint64_t)ri.w << 32);
    edges[e] = make_uint4((uint32_t)t, ri.x, ri.y, T >= (1ull << 53) ? 0xffffffffu : (uint32_t)(T >> 21));
  }
}

// Weighted edge records (64 bytes): the header above, then the high words
// (bits 32..52) of the target's slot thresholds B_0 .. B_11 (unused entries
// all ones).
__global__ void k_edge_records_w(int64_t nnz, const int32_t* __restrict__ colidx, const uint4* __restrict__ rowinfo,
                                 const uint64_t* __restrict__ B, uint4* __restrict__ edges) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = colidx[e];
    const uint4 ri = rowinfo[t];
    const uint64_t T = (uint64_t)ri.z | ((uint64_t)ri.w << 32);
    uint32_t h[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) h[j] = (uint32_t)j + 1u < ri.y ? (uint32_t)(B[(size_t)ri.x + j] >> 32) : 0xffffffffu;
    uint4* r = edges + (size_t)e * 4;
    r[0] = make_uint4((uint32_t)t, ri.x, ri.y, T >= (1ull << 53) ? 0xffffffffu : (uint32_t)(T >> 21));
    r[1] = make_uint4(h[0], h[1], h[2], h[3]);
    r[2] = make_uint4(h[4], h[5], h[6], h[7]);
    r[3] = make_uint4(h[8], h[9], h[10], h[11]);
  }
}

void free_graph_arrays(fc_graph* g, cudaStream_t st) {
  void* ptrs[] = {g->rowptr, g->colidx, g->w, g->deg, g->dw, g->S, g->order, g->rowinfo, g->B, g->edges,
                  g->alphas_d, g->d_err, g->d_counter, g->d_stats, g->voff, g->gid, g->alpha_v,
                  g->gorder, g->item_ns, g->t0_ns, g->bpar, g->binv, g->bdepth};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, st);
  if (g->ws) cudaFree(g->ws);
  if (g->sv) cudaFree(g->sv);
}

}  // namespace fcx

using namespace fcx;

extern "C" const char* fc_status_str(fc_status s) {
  switch (s) {
    case FC_OK: return "ok";
    case FC_EINVAL: return "invalid argument or input graph";
    case FC_ENOMEM: return "out of memory";
    case FC_ECUDA: return "CUDA error";
    case FC_ENOCONV: return "solver did not converge";
    case FC_ETIMEOUT: return "sampler watchdog expired";
    case FC_EOVERFLOW: return "visit counter overflow";
  }
  return "unknown status";
}

extern "C" const char* fc_last_error_message(void) { return g_last_error.c_str(); }

extern "C" uint64_t fc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" fc_status fc_release_scratch(void) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  for (auto& sc : g_scratch) {
    if (sc.ptr) {
      FC_CK(cudaDeviceSynchronize());
      FC_CK(cudaFree(sc.ptr));
      sc.ptr = nullptr;
      sc.bytes = 0;
    }
  }
  return FC_OK;
}

#define BUILD_CK(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      fc_status s_ = cuda_fail(e_, #call);               \
      free_graph_arrays(g, st);                          \
      delete g;                                          \
      return s_;                                         \
    }                                                    \
  } while (0)

fc_status fcx::build_impl(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx, const float* w,
                          const double* alphas, int32_t n_alpha, uint32_t flags, void* stream, fc_graph** out,
                          int32_t G, const int64_t* voff_h, const double* galpha_h, int32_t root) {
  if (out == nullptr) return fcx::invalid("fc_build_augmented / fc_build_batch: null output pointer");
  *out = nullptr;
  if (n < 1 || n >= (1 << 30) || nnz < 0 || nnz >= (int64_t(1) << 32) || n_alpha < 1 || n_alpha > 64 ||
      rowptr == nullptr || (nnz > 0 && colidx == nullptr) || alphas == nullptr ||
      (flags != FC_HOST_PTRS && flags != FC_DEVICE_PTRS)) {
    set_error("fc_build_augmented: argument out of range");
    return FC_EINVAL;
  }
  for (int i = 0; i < n_alpha; ++i) {
    if (!(std::isfinite(alphas[i]) && alphas[i] > 0.0)) {
      set_error("fc_build_augmented: alpha must be finite and > 0");
      return FC_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  fc_graph* g = new fc_graph();
  g->n = n;
  g->nnz = nnz;
  g->n_alpha = n_alpha;
  g->weighted = (w != nullptr);
  g->alphas.assign(alphas, alphas + n_alpha);
  g->root = root;
  BUILD_CK(cudaGetDevice(&g->device));
  {
    size_t freeb = 0;
    BUILD_CK(cudaMemGetInfo(&freeb, &g->device_bytes));
  }
  retain_pool(g->device);
  if (G > 0) {
    g->num_graphs = G;
    g->voff_h.assign(voff_h, voff_h + G + 1);
    g->galpha.assign(galpha_h, galpha_h + G);
    std::vector<int32_t> ord(G);
    for (int i = 0; i < G; ++i) {
      ord[i] = i;
      g->max_ng = std::max<int32_t>(g->max_ng, (int32_t)(voff_h[i + 1] - voff_h[i]));
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      return (voff_h[a + 1] - voff_h[a]) > (voff_h[b + 1] - voff_h[b]);
    });
    BUILD_CK(cudaMallocAsync((void**)&g->voff, (G + 1) * sizeof(int64_t), st));
    BUILD_CK(cudaMallocAsync((void**)&g->gorder, G * sizeof(int32_t), st));
    BUILD_CK(cudaMallocAsync((void**)&g->gid, (size_t)n * sizeof(int32_t), st));
    BUILD_CK(cudaMallocAsync((void**)&g->alpha_v, (size_t)n * sizeof(double), st));
    BUILD_CK(cudaMallocAsync((void**)&g->t0_ns, sizeof(unsigned long long), st));
    double* galpha_d = nullptr;
    BUILD_CK(cudaMallocAsync((void**)&galpha_d, G * sizeof(double), st));
    BUILD_CK(cudaMemcpyAsync(g->voff, voff_h, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    BUILD_CK(cudaMemcpyAsync(g->gorder, ord.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    BUILD_CK(cudaMemcpyAsync(galpha_d, galpha_h, G * sizeof(double), cudaMemcpyHostToDevice, st));
    k_batch_vertex<<<grid_for(n, 256), 256, 0, st>>>(n, G, g->voff, galpha_d, g->gid, g->alpha_v, nullptr);
    BUILD_CK((fcx::note_launch(), cudaGetLastError()));
    BUILD_CK(cudaFreeAsync(galpha_d, st));
    // ord must outlive the async copy
    BUILD_CK(cudaStreamSynchronize(st));
  }
  const size_t nz = (size_t)(nnz > 0 ? nnz : 1);
  BUILD_CK(cudaMallocAsync((void**)&g->rowptr, (n + 1) * sizeof(int64_t), st));
  BUILD_CK(cudaMallocAsync((void**)&g->colidx, nz * sizeof(int32_t), st));
  if (g->weighted) {
    BUILD_CK(cudaMallocAsync((void**)&g->w, nz * sizeof(float), st));
    BUILD_CK(cudaMallocAsync((void**)&g->S, nz * sizeof(double), st));
    BUILD_CK(cudaMallocAsync((void**)&g->B, nz * n_alpha * sizeof(uint64_t), st));
  }
  BUILD_CK(cudaMallocAsync((void**)&g->deg, n * sizeof(int32_t), st));
  BUILD_CK(cudaMallocAsync((void**)&g->dw, n * sizeof(double), st));
  BUILD_CK(cudaMallocAsync((void**)&g->order, n * sizeof(int32_t), st));
  BUILD_CK(cudaMallocAsync((void**)&g->rowinfo, (size_t)n * n_alpha * sizeof(uint4), st));
  BUILD_CK(cudaMallocAsync((void**)&g->alphas_d, n_alpha * sizeof(double), st));
  BUILD_CK(cudaMallocAsync((void**)&g->d_err, 4 * sizeof(uint32_t), st));
  BUILD_CK(cudaMallocAsync((void**)&g->d_counter, 2 * sizeof(unsigned long long), st));
  BUILD_CK(cudaMallocAsync((void**)&g->d_stats, 16 * sizeof(unsigned long long), st));

  const cudaMemcpyKind kind = flags == FC_DEVICE_PTRS ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  BUILD_CK(cudaMemcpyAsync(g->rowptr, rowptr, (n + 1) * sizeof(int64_t), kind, st));
  if (nnz > 0) BUILD_CK(cudaMemcpyAsync(g->colidx, colidx, nnz * sizeof(int32_t), kind, st));
  if (g->weighted && nnz > 0) BUILD_CK(cudaMemcpyAsync(g->w, w, nnz * sizeof(float), kind, st));
  BUILD_CK(cudaMemcpyAsync(g->alphas_d, alphas, n_alpha * sizeof(double), cudaMemcpyHostToDevice, st));
  BUILD_CK(cudaMemsetAsync(g->d_err, 0, 4 * sizeof(uint32_t), st));

  k_validate<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, nnz, g->rowptr, g->colidx, g->w, g->gid,
                                                              g->d_err);
  BUILD_CK((fcx::note_launch(), cudaGetLastError()));
  uint32_t hs[4] = {0, 0, 0, 0};
  BUILD_CK(cudaMemcpyAsync(hs, g->d_err, sizeof(hs), cudaMemcpyDeviceToHost, st));
  BUILD_CK(cudaStreamSynchronize(st));
  if (hs[0] != 0) {
    set_error("fc_build_augmented: CSR violates the input contract (range, sorted rows, no self-loops/"
              "duplicates, symmetry, finite non-negative weights)");
    free_graph_arrays(g, st);
    cudaStreamSynchronize(st);
    delete g;
    return FC_EINVAL;
  }
  // rowptr is now known to be in range and monotone
  k_degrees<<<grid_for(n, 256), 256, 0, st>>>(n, g->rowptr, g->w, g->deg, g->dw, g->S,
                                              (int32_t*)(g->d_err + 1));
  BUILD_CK((fcx::note_launch(), cudaGetLastError()));
  BUILD_CK(cudaMemcpyAsync(hs, g->d_err, sizeof(hs), cudaMemcpyDeviceToHost, st));
  BUILD_CK(cudaStreamSynchronize(st));
  g->max_deg = (int32_t)hs[1];
  BUILD_CK(cudaMemsetAsync(g->d_err, 0, 4 * sizeof(uint32_t), st));

  // ascending-degree order, ties by id (stable LSD radix sort)
  {
    const int32_t nblk = (int32_t)((n + RS_TILE - 1) / RS_TILE);
    uint32_t *k0 = nullptr, *k1 = nullptr, *hist = nullptr, *offs = nullptr;
    int32_t* v1 = nullptr;
    BUILD_CK(cudaMallocAsync((void**)&k0, n * sizeof(uint32_t), st));
    BUILD_CK(cudaMallocAsync((void**)&k1, n * sizeof(uint32_t), st));
    BUILD_CK(cudaMallocAsync((void**)&v1, n * sizeof(int32_t), st));
    BUILD_CK(cudaMallocAsync((void**)&hist, (size_t)256 * nblk * sizeof(uint32_t), st));
    BUILD_CK(cudaMallocAsync((void**)&offs, (size_t)256 * nblk * sizeof(uint32_t), st));
    k_iota_keys<<<grid_for(n, 256), 256, 0, st>>>(n, g->deg, k0, g->order);
    BUILD_CK((fcx::note_launch(), cudaGetLastError()));
    int passes = 1;
    while (passes < 4 && (uint32_t)g->max_deg >> (8 * passes)) ++passes;
    uint32_t* kin = k0;
    uint32_t* kout = k1;
    int32_t* vin = g->order;
    int32_t* vout = v1;
    for (int p = 0; p < passes; ++p) {
      k_rs_hist<<<nblk, 32, 0, st>>>(n, kin, 8 * p, hist, nblk);
      BUILD_CK((fcx::note_launch(), cudaGetLastError()));
      fc_status r = exclusive_scan(hist, offs, (int64_t)256 * nblk, st);
      if (r != FC_OK) {
        free_graph_arrays(g, st);
        delete g;
        return r;
      }
      k_rs_scatter<<<nblk, 32, 0, st>>>(n, kin, vin, kout, vout, 8 * p, offs, nblk);
      BUILD_CK((fcx::note_launch(), cudaGetLastError()));
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    if (g->num_graphs > 0) {
      // second stable pass: by graph, so each graph's start vertices are contiguous
      k_gid_keys<<<grid_for(n, 256), 256, 0, st>>>(n, vin, g->gid, kin);
      BUILD_CK((fcx::note_launch(), cudaGetLastError()));
      for (int pass = 0; pass < 4 && ((uint32_t)(g->num_graphs - 1) >> (8 * pass)); ++pass) {
        k_rs_hist<<<nblk, 32, 0, st>>>(n, kin, 8 * pass, hist, nblk);
        BUILD_CK((fcx::note_launch(), cudaGetLastError()));
        fc_status r = exclusive_scan(hist, offs, (int64_t)256 * nblk, st);
        if (r != FC_OK) {
          free_graph_arrays(g, st);
          delete g;
          return r;
        }
        k_rs_scatter<<<nblk, 32, 0, st>>>(n, kin, vin, kout, vout, 8 * pass, offs, nblk);
        BUILD_CK((fcx::note_launch(), cudaGetLastError()));
        std::swap(kin, kout);
        std::swap(vin, vout);
      }
    }
    if (vin != g->order)
      BUILD_CK(cudaMemcpyAsync(g->order, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    BUILD_CK(cudaFreeAsync(k0, st));
    BUILD_CK(cudaFreeAsync(k1, st));
    BUILD_CK(cudaFreeAsync(v1, st));
    BUILD_CK(cudaFreeAsync(hist, st));
    BUILD_CK(cudaFreeAsync(offs, st));
  }

  for (int a = 0; a < n_alpha; ++a) {
    const double gamma = root >= 0 ? 0.0 : 1.0;
    k_thr_vertex<<<grid_for(n, 256), 256, 0, st>>>(n, g->alphas[a], g->alpha_v, g->weighted, g->rowptr,
                                                   g->deg, g->dw, gamma, root, g->rowinfo + (size_t)a * n);
    BUILD_CK((fcx::note_launch(), cudaGetLastError()));
    if (g->weighted && nnz > 0) {
      k_thr_nnz<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(n, g->alphas[a], g->alpha_v, g->rowptr, g->S,
                                                                g->dw, gamma, g->B + (size_t)a * nnz);
      BUILD_CK((fcx::note_launch(), cudaGetLastError()));
    }
  }
  unsigned long long* d_local = nullptr;
  unsigned long long h_local = 0;
  if (nnz > 0) {
    BUILD_CK(cudaMallocAsync((void**)&d_local, sizeof(unsigned long long), st));
    BUILD_CK(cudaMemsetAsync(d_local, 0, sizeof(unsigned long long), st));
    k_id_locality<<<(unsigned)(((nnz + LOC_RUN - 1) / LOC_RUN + 255) / 256), 256, 0, st>>>(n, nnz, g->rowptr,
                                                                                       g->colidx, d_local);
    BUILD_CK((fcx::note_launch(), cudaGetLastError()));
    BUILD_CK(cudaMemcpyAsync(&h_local, d_local, sizeof(h_local), cudaMemcpyDeviceToHost, st));
    BUILD_CK(cudaFreeAsync(d_local, st));
    const size_t rec = g->weighted ? 4 : 1;  // uint4 per record
    BUILD_CK(cudaMallocAsync((void**)&g->edges, (size_t)nnz * n_alpha * rec * sizeof(uint4), st));
    for (int a = 0; a < n_alpha; ++a) {
      if (g->weighted)
        k_edge_records_w<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, g->colidx, g->rowinfo + (size_t)a * n,
                                                            g->B + (size_t)a * nnz, g->edges + (size_t)a * nnz * 4);
      else
        k_edge_records<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, g->colidx, g->rowinfo + (size_t)a * n,
                                                          g->edges + (size_t)a * nnz);
      BUILD_CK((fcx::note_launch(), cudaGetLastError()));
    }
  }
  BUILD_CK(cudaStreamSynchronize(st));
  g->id_local = nnz > 0 && h_local * 4 > (unsigned long long)nnz;
  *out = g;
  return FC_OK;
}

extern "C" fc_status fc_build_augmented(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                        const float* w, const double* alphas, int32_t n_alpha, uint32_t flags,
                                        void* stream, fc_graph** out) {
  return build_impl(n, nnz, rowptr, colidx, w, alphas, n_alpha, flags, stream, out, 0, nullptr, nullptr, -1);
}

extern "C" fc_status fc_build_batch(int32_t num_graphs, const int64_t* vertex_offsets, int64_t nnz,
                                    const int64_t* rowptr, const int32_t* colidx, const float* w,
                                    const double* graph_alphas, uint32_t flags, void* stream, fc_graph** out) {
  if (out == nullptr) return fcx::invalid("fc_build_batch: bad argument");
  *out = nullptr;
  if (num_graphs < 1 || vertex_offsets == nullptr || graph_alphas == nullptr || vertex_offsets[0] != 0) {
    set_error("fc_build_batch: bad argument");
    return FC_EINVAL;
  }
  for (int32_t i = 0; i < num_graphs; ++i) {
    if (vertex_offsets[i + 1] <= vertex_offsets[i] || !(std::isfinite(graph_alphas[i]) && graph_alphas[i] > 0.0)) {
      set_error("fc_build_batch: graphs must be non-empty and alphas finite and > 0");
      return FC_EINVAL;
    }
  }
  const int64_t n = vertex_offsets[num_graphs];
  if (n >= (1 << 30)) {
    set_error("fc_build_batch: too many vertices");
    return FC_EINVAL;
  }
  const double one = 1.0;
  return build_impl((int32_t)n, nnz, rowptr, colidx, w, &one, 1, flags, stream, out, num_graphs, vertex_offsets,
                    graph_alphas, -1);
}

extern "C" fc_status fc_graph_info(const fc_graph* g, int32_t* n, int64_t* nnz, int32_t* n_alpha,
                                   int32_t* weighted) {
  if (g == nullptr) return fcx::invalid("fc_graph_info: bad argument");
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (n_alpha) *n_alpha = g->n_alpha;
  if (weighted) *weighted = g->weighted ? 1 : 0;
  return FC_OK;
}

extern "C" fc_status fc_set_sampler_shape(fc_graph* g, int32_t walkers_per_tree, int32_t max_trees_resident,
                                          int32_t smem, int32_t regs) {
  if (g == nullptr || walkers_per_tree < 0 || walkers_per_tree > 1024 || (walkers_per_tree % 32) != 0 ||
      max_trees_resident < 0 || smem < 0 || smem > 2 ||
      !(regs == 0 || regs == 32 || regs == 40 || regs == 48 || regs == 64))
    return fcx::invalid("fc_set_sampler_shape: bad argument");
  g->walkers = walkers_per_tree;
  g->max_trees = max_trees_resident;
  g->smem_mode = smem;
  g->regs = regs;
  return FC_OK;
}

extern "C" fc_status fc_set_start_order(fc_graph* g, int32_t order) {
  if (g == nullptr || order < 0 || order > 4) return fcx::invalid("fc_set_start_order: bad argument");
  g->order_auto = order == 4;
  g->order_desc = order == 4 ? 0 : (order & 1);
  g->order_id = order == 4 ? 0 : (order >> 1);
  return FC_OK;
}

extern "C" fc_status fc_set_sampler_kernel(fc_graph* g, int32_t kernel) {
  if (g == nullptr || kernel < 0 || kernel > 2) return fcx::invalid("fc_set_sampler_kernel: bad argument");
  if (kernel == 2 && g->edges == nullptr) {
    set_error("fc_set_sampler_kernel: edge records exist only for graphs with edges");
    return FC_EINVAL;
  }
  g->kernel_pref = kernel;
  return FC_OK;
}

extern "C" int32_t fc_sampler_last_kernel(const fc_graph* g) { return g ? g->last_kernel : -1; }

extern "C" fc_status fc_set_sampler_cluster(fc_graph* g, int32_t ctas_per_tree) {
  if (g == nullptr || !(ctas_per_tree == 0 || ctas_per_tree == 1 || ctas_per_tree == 2 || ctas_per_tree == 4 ||
                        ctas_per_tree == 8))
    return fcx::invalid("fc_set_sampler_cluster: bad argument");
  g->cluster = ctas_per_tree;
  return FC_OK;
}

extern "C" int32_t fc_sampler_last_cluster(const fc_graph* g) { return g ? g->last_cluster : -1; }

extern "C" fc_status fc_set_sampler_bitmap(fc_graph* g, int32_t mode) {
  if (g == nullptr || mode < 0 || mode > 3) return fcx::invalid("fc_set_sampler_bitmap: bad argument");
  g->bitmap_mode = mode;
  return FC_OK;
}

extern "C" fc_status fc_set_sampler_pops(fc_graph* g, int32_t mode) {
  if (g == nullptr || mode < 0 || mode > 2) return fcx::invalid("fc_set_sampler_pops: bad argument");
  g->pops_mode = mode;
  return FC_OK;
}

extern "C" fc_status fc_sampler_last_shape(const fc_graph* g, int32_t* walkers_per_tree, int32_t* regs,
                                           int32_t* ctas) {
  if (g == nullptr) return fcx::invalid("fc_sampler_last_shape: bad argument");
  if (walkers_per_tree) *walkers_per_tree = g->last_W;
  if (regs) *regs = g->last_regs;
  if (ctas) *ctas = g->last_grid;
  return FC_OK;
}

extern "C" void fc_destroy(fc_graph* g) {
  if (g == nullptr) return;
  cudaStream_t st = 0;
  cudaDeviceSynchronize();
  free_graph_arrays(g, st);
  cudaStreamSynchronize(st);
  delete g;
}

extern "C" int64_t fc_tau_for(double eps, double delta, double kappa, int64_t m) {
  if (!(eps > 0 && eps < 1 && delta > 0 && delta < 1 && kappa > 0 && kappa < 1 && m >= 1)) return -1;
  const double e = (1.0 - kappa) * eps;
  return (int64_t)std::ceil(std::log(2.0 * (double)m / delta) / (2.0 * e * e));
}
