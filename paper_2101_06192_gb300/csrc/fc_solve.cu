// Linear solves in A = I + alpha L (the matrix of the grounded pivot system of
// Algorithm 1, and of the CG ground truth of Sec. 6.1), and in the Laplacian
// L of a connected G itself (the pivot column of L^+ that the electrical-
// closeness algorithm of Sec. 3 needs): A = sigma I + alpha L, sigma 1 or 0.
//
// Mixed precision: the outer loop is iterative refinement in FP64
// (r = b - A x with FP64 x and FP64 arithmetic, x += correction); the
// correction solves A d = r / ||r|| with Jacobi-preconditioned CG in FP32.
// Several right-hand sides run side by side (column j of an [m][n] block),
// each with its own CG scalars; reductions are two-pass and fixed-order, so
// results do not depend on scheduling.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fc_internal.cuh"

namespace cgr = cooperative_groups;

namespace fcx {

constexpr int SV_T = 256;

// Rows are processed by groups of RG consecutive lanes (strided over the
// row's entries, then a shuffle reduction), so long rows do not serialise one
// thread.  Each block covers SV_T / RG rows.
constexpr int RG = 8;
constexpr int ROWS_PER_BLOCK = SV_T / RG;

__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = RG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Block-wide sum of two doubles (warp shuffles, then one warp); the result
// is valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double wa[SV_T / 32], wb[SV_T / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    wa[threadIdx.x >> 5] = a;
    wb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0.0;
    b = 0.0;
    for (int w = 0; w < SV_T / 32; ++w) {
      a += wa[w];
      b += wb[w];
    }
  }
}

__device__ __forceinline__ float group_sumf(float v) {
#pragma unroll
  for (int o = RG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- FP64 residual r = b - A x, partial sums of r.r and b.b ---------------
__global__ void k_resid64(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                          const float* __restrict__ w, const double* __restrict__ dw, double sigma, double alpha,
                          const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
                          double* __restrict__ prr, double* __restrict__ pbb, int nb) {
  // blocks stride over the chunks of ROWS_PER_BLOCK rows; nb = gridDim.x partials per column
  const int j = blockIdx.y;
  const int gl = threadIdx.x % RG;
  const size_t off = (size_t)j * n;
  double rr = 0.0, bb = 0.0;
  for (int64_t c = blockIdx.x; c * ROWS_PER_BLOCK < n; c += gridDim.x) {
    const int64_t v = c * ROWS_PER_BLOCK + threadIdx.x / RG;
    double acc = 0.0;
    if (v < n) {
      for (int64_t e = rowptr[v] + gl; e < rowptr[v + 1]; e += RG) {
        const double we = w ? (double)w[e] : 1.0;
        acc += we * x[off + colidx[e]];
      }
    }
    acc = group_sum(acc);
    if (v < n && gl == 0) {
      const double ax = x[off + v] * (sigma + alpha * dw[v]) - alpha * acc;
      const double rv = b[off + v] - ax;
      r[off + v] = rv;
      rr += rv * rv;
      bb += b[off + v] * b[off + v];
    }
  }
  block_sum2(rr, bb);
  if (threadIdx.x == 0) {
    prr[(size_t)j * nb + blockIdx.x] = rr;
    pbb[(size_t)j * nb + blockIdx.x] = bb;
  }
}

__global__ void k_colsum(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double red[SV_T];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += SV_T) s += part[(size_t)j * nb + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = SV_T / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

// ---- FP32 inner PCG ---------------------------------------------------------
struct Inner {
  float* r;   // residual of the correction system
  float* p;
  float* q;
  float* d;   // correction
  double* scal;  // per column: [0] rz, [1] pq, [2] rz_new, [3] rr, [4] scale, [5] active
};

// r32 = r64 * inv_scale; d = 0; p = z = r32 / diag; partial r.z and r.r
__global__ void k_inner_init(int32_t n, const double* __restrict__ r64, const float* __restrict__ prec,
                             const double* __restrict__ scal, Inner in, double* __restrict__ prz,
                             double* __restrict__ prr, int nb) {
  const int j = blockIdx.y;
  const size_t off = (size_t)j * n;
  const double sc = scal[j * 8 + 4];
  float rzf = 0.0f, rrf = 0.0f;  // per-thread partials in FP32, then FP64 across threads
  for (int64_t v = (int64_t)blockIdx.x * SV_T + threadIdx.x; v < n; v += (int64_t)gridDim.x * SV_T) {
    const float rv = (float)(r64[off + v] * sc);
    const float z = prec ? rv * prec[v] : rv;
    in.r[off + v] = rv;
    in.p[off + v] = z;
    in.d[off + v] = 0.0f;
    rzf = fmaf(rv, z, rzf);
    rrf = fmaf(rv, rv, rrf);
  }
  double rz = rzf, rr = rrf;
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    prz[(size_t)j * nb + blockIdx.x] = rz;
    prr[(size_t)j * nb + blockIdx.x] = rr;
  }
}

// q = A p (FP32), partial p.q
__global__ void k_spmv_pq(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                          const float* __restrict__ w, const float* __restrict__ diag32, float alpha, Inner in,
                          double* __restrict__ ppq, int nb) {
  const int j = blockIdx.y;
  const int gl = threadIdx.x % RG;
  const size_t off = (size_t)j * n;
  const float* pj = in.p + off;
  float pqf = 0.0f;
  for (int64_t c = blockIdx.x; c * ROWS_PER_BLOCK < n; c += gridDim.x) {
    const int64_t v = c * ROWS_PER_BLOCK + threadIdx.x / RG;
    float acc = 0.0f;
    if (v < n) {
      for (int64_t e = rowptr[v] + gl; e < rowptr[v + 1]; e += RG) acc += (w ? w[e] : 1.0f) * pj[colidx[e]];
    }
    acc = group_sumf(acc);
    if (v < n && gl == 0) {
      const float pv = pj[v];
      const float qv = pv * diag32[v] - alpha * acc;
      in.q[off + v] = qv;
      pqf = fmaf(pv, qv, pqf);
    }
  }
  double pq = pqf, unused = 0.0;
  block_sum2(pq, unused);
  if (threadIdx.x == 0) ppq[(size_t)j * nb + blockIdx.x] = pq;
}

// d += a p; r -= a q; partial r.z, r.r with z = r / diag
__global__ void k_inner_update(int32_t n, const float* __restrict__ prec, const double* __restrict__ scal,
                               Inner in, double* __restrict__ prz, double* __restrict__ prr, int nb) {
  const int j = blockIdx.y;
  const size_t off = (size_t)j * n;
  const double* sc = scal + j * 8;
  const float a = (sc[5] != 0.0 && sc[1] != 0.0) ? (float)(sc[0] / sc[1]) : 0.0f;
  float rzf = 0.0f, rrf = 0.0f;
  for (int64_t v = (int64_t)blockIdx.x * SV_T + threadIdx.x; v < n; v += (int64_t)gridDim.x * SV_T) {
    in.d[off + v] += a * in.p[off + v];
    const float rv = in.r[off + v] - a * in.q[off + v];
    in.r[off + v] = rv;
    const float z = prec ? rv * prec[v] : rv;
    rzf = fmaf(rv, z, rzf);
    rrf = fmaf(rv, rv, rrf);
  }
  double rz = rzf, rr = rrf;
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    prz[(size_t)j * nb + blockIdx.x] = rz;
    prr[(size_t)j * nb + blockIdx.x] = rr;
  }
}

// p = z + beta p with beta = rz_new / rz
__global__ void k_inner_p(int32_t n, const float* __restrict__ prec, const double* __restrict__ scal, Inner in) {
  const int j = blockIdx.y;
  const size_t off = (size_t)j * n;
  const double* sc = scal + j * 8;
  const float beta = sc[0] != 0.0 ? (float)(sc[2] / sc[0]) : 0.0f;
  for (int64_t v = (int64_t)blockIdx.x * SV_T + threadIdx.x; v < n; v += (int64_t)gridDim.x * SV_T) {
    const float z = prec ? in.r[off + v] * prec[v] : in.r[off + v];
    in.p[off + v] = z + beta * in.p[off + v];
  }
}

// scalar bookkeeping after k_inner_update: rz <- rz_new (done after k_inner_p
// has used both), rr stored
// scal[j][f + i] = sums[i m + j] for i < cnt: the per-column scalars from
// the column sums (one launch instead of a strided copy of m 8-byte rows,
// which costs about a microsecond per row)
__global__ void k_put_scal(int m, const double* __restrict__ sums, int f, int cnt, double* __restrict__ scal) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m)
    for (int i = 0; i < cnt; ++i) scal[j * 8 + f + i] = sums[(size_t)i * m + j];
}

__global__ void k_scal_shift(int m, double* scal) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) scal[j * 8 + 0] = scal[j * 8 + 2];
}

// x += (1/scale) d (FP64), only for active columns
__global__ void k_correct(int32_t n, const double* __restrict__ scal, const float* __restrict__ d,
                          double* __restrict__ x) {
  const int j = blockIdx.y;
  const double* sc = scal + j * 8;
  if (sc[5] == 0.0) return;
  const size_t off = (size_t)j * n;
  for (int64_t v = (int64_t)blockIdx.x * SV_T + threadIdx.x; v < n; v += (int64_t)gridDim.x * SV_T)
    x[off + v] += (double)d[off + v] / sc[4];
}

// the FP32 diagonal and its reciprocal (the Jacobi preconditioner, applied
// as a product)
__global__ void k_diag32(int32_t n, const double* __restrict__ dw, double sigma, double alpha,
                         float* __restrict__ diag32, float* __restrict__ inv32) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) {
    const double d = sigma + alpha * dw[v];
    diag32[v] = (float)d;
    inv32[v] = (float)(1.0 / d);
  }
}

__global__ void k_fill(int64_t len, double val, double* __restrict__ a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) a[i] = val;
}

// x over V' (n+1 entries, x[n] = x(u*) = 0 on entry) -> mean-zero gauge
__global__ void k_shift(int64_t len, const double* __restrict__ sum, double* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) x[i] -= *sum / (double)len;
}

__global__ void k_partial_sum(int64_t len, const double* __restrict__ a, double* __restrict__ part) {
  __shared__ double red[SV_T];
  const int64_t i = (int64_t)blockIdx.x * SV_T + threadIdx.x;
  red[threadIdx.x] = i < len ? a[i] : 0.0;
  __syncthreads();
  for (int s = SV_T / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}


// Singular systems (sigma = 0, L of a connected graph): the residual's
// component along 1 lies in L's kernel, where CG cannot reduce it; rounding
// in the FP64 residual leaves a little there, so each refinement step
// projects it out.  One block per column (fixed-order sums): r_j -= mean(r_j)
// and rr[j] = |r_j|^2 after the projection.  il: element (v, j) at v m + j,
// else at j n + v.
__global__ void k_proj_mean(int32_t n, int m, bool il, double* __restrict__ r, double* __restrict__ rr) {
  __shared__ double red[SV_T];
  const int j = blockIdx.x;
  auto at = [&](int64_t v) -> double& { return r[il ? (size_t)v * m + j : (size_t)j * n + v]; };
  double s = 0.0;
  for (int64_t v = threadIdx.x; v < n; v += SV_T) s += at(v);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = SV_T / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  const double mean = red[0] / (double)n;
  __syncthreads();
  double q = 0.0;
  for (int64_t v = threadIdx.x; v < n; v += SV_T) {
    const double x = at(v) - mean;
    at(v) = x;
    q += x * x;
  }
  red[threadIdx.x] = q;
  __syncthreads();
  for (int k = SV_T / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) rr[j] = red[0];
}

// ---------------------------------------------------------------------------
// One right-hand side.
//
// Sums over rows, s_v = sum_j w_vj x_j, in edge tiles: tile t holds the
// entries [t TL, (t+1) TL) of the CSR arrays and is one warp, TL_E
// consecutive entries per lane, whatever the rows.  A row of a few thousand
// entries (the hubs of a scale-free graph) is spread over many lanes and
// warps instead of serialising one group of lanes, and every lane issues TL_E
// independent gathers.  Within a tile a segmented scan over the lanes' last
// rows (keys nondecreasing) joins rows that cross lanes; a row that crosses
// tiles leaves one partial per tile (tail[t0] in the tile where it starts,
// head[t] in each later tile) and is summed from them in tile order.  Tiles
// need no block barrier, so the warps of a block hide each other's memory
// latency.  Every addition has a fixed place, so results do not depend on
// scheduling.
// ---------------------------------------------------------------------------
constexpr int TL_T = 32;              // lanes per tile (one warp)
constexpr int TL_E = 8;               // entries per lane
constexpr int TL = TL_T * TL_E;       // entries per tile
constexpr int TL_RCAP = TL + 2;       // row offsets staged in shared memory (general tiles)
constexpr int TL_W = SV_T / 32;       // tiles in flight per block

// row0[t] / row1[t]: the rows holding the first / last entry of tile t (the
// largest v with rowptr[v] <= e)
__global__ void k_tile_rows(int32_t n, int64_t nnz, const int64_t* __restrict__ rowptr, int64_t ntiles,
                            int32_t* __restrict__ row0, int32_t* __restrict__ row1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * ntiles) return;
  const int64_t t = i >> 1;
  const int64_t e = (i & 1) ? std::min<int64_t>((t + 1) * TL, nnz) - 1 : t * TL;
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int32_t mid = lo + (hi - lo + 1) / 2;
    if (rowptr[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  ((i & 1) ? row1 : row0)[t] = lo;
}

// Per-thread tile metadata, one word per thread, fixed for the whole solve:
//   bit j (1..TL_E-1)  entry j of the thread starts a new row
//   bit TM_EL          the thread's last row ends at its last entry
//   bits TM_RF..       the row of its first entry, relative to row0[t]
//   TM_BEFORE          the tile's first row began in an earlier tile
//   TM_GENERAL         the tile has empty rows between its first and last
//                      row: walked through the row offsets instead
constexpr uint32_t TM_EL = 1u << TL_E;
constexpr int TM_RF = TL_E + 1;
constexpr uint32_t TM_RF_MASK = 0xFFFu;
constexpr uint32_t TM_BEFORE = 1u << 29;
constexpr uint32_t TM_GENERAL = 1u << 30;

__global__ void __launch_bounds__(SV_T) k_tile_meta(int64_t nnz, const int64_t* __restrict__ rowptr, int64_t ntiles,
                                                    const int32_t* __restrict__ row0,
                                                    const int32_t* __restrict__ row1, uint32_t* __restrict__ meta) {
  const int lane = threadIdx.x & 31;
  for (int64_t t = (int64_t)blockIdx.x * TL_W + (threadIdx.x >> 5); t < ntiles; t += (int64_t)gridDim.x * TL_W) {
    const int64_t E0 = t * TL;
    const int ne = (int)std::min<int64_t>(TL, nnz - E0);
    const int32_t rs = row0[t];
    const int nr = row1[t] - rs + 1;
    int empty = 0;
    for (int i = 1 + lane; i < nr; i += TL_T) empty |= rowptr[rs + i + 1] == rowptr[rs + i];
    const bool general = __any_sync(0xffffffffu, empty) != 0;
    uint32_t mw = (general ? TM_GENERAL : 0u) | (rowptr[rs] < E0 ? TM_BEFORE : 0u);
    const int le0 = lane * TL_E;
    const int cnt = ne - le0 >= TL_E ? TL_E : (ne - le0 > 0 ? ne - le0 : 0);
    if (!general && cnt > 0) {
      int lo = 0, hi = nr - 1;  // the row holding entry le0
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rowptr[rs + mid] - E0 <= le0) lo = mid;
        else hi = mid - 1;
      }
      mw |= (uint32_t)lo << TM_RF;
      int cur = lo;
      int64_t nxt = rowptr[rs + cur + 1] - E0;
      for (int j = 1; j < cnt; ++j)
        if (nxt == le0 + j) {  // no empty rows here: one row per boundary
          mw |= 1u << j;
          ++cur;
          nxt = rowptr[rs + cur + 1] - E0;
        }
      if (nxt == le0 + cnt) mw |= TM_EL;
    }
    meta[t * TL_T + lane] = mw;
  }
}

struct TileSmem {
  int32_t off[TL_W][TL_RCAP];  // rowptr[row0 + i] - t TL (general tiles), one row per warp
};

template <typename V>
struct TileArgs {
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* colidx;
  const float* w;
  const int32_t* row0;
  const int32_t* row1;
  const uint32_t* meta;  // [tiles][TL_T] from k_tile_meta
  const uint32_t* span;  // bit v: row v is empty or crosses tiles (s[v] not written)
  V* s;     // rows inside one tile
  V* head;  // [tiles] partial of the tile's first row if it began earlier
  V* tail;  // [tiles] partial of the tile's last row if it began here and goes on
  bool vec; // colidx / w 16-byte aligned: vector loads for full tiles
};

// What a lane needs of one tile before its gathers, loaded one tile ahead.
struct TileIn {
  int32_t col[TL_E];
  uint32_t mw;
  int32_t rs;
};

template <typename V>
__device__ __forceinline__ void tile_load(const TileArgs<V>& a, int64_t t, TileIn& ti) {
  const int lane = threadIdx.x & 31;
  const int64_t E0 = t * TL;
  const int ne = (int)std::min<int64_t>(TL, a.nnz - E0);
  const int le0 = lane * TL_E;
  const int cnt = ne - le0 >= TL_E ? TL_E : (ne - le0 > 0 ? ne - le0 : 0);
  ti.rs = a.row0[t];
  ti.mw = a.meta[t * TL_T + lane];
  if (a.vec && ne == TL) {
    const int4* c4 = reinterpret_cast<const int4*>(a.colidx + E0 + le0);
    const int4 c0 = c4[0], c1 = c4[1];
    ti.col[0] = c0.x; ti.col[1] = c0.y; ti.col[2] = c0.z; ti.col[3] = c0.w;
    ti.col[4] = c1.x; ti.col[5] = c1.y; ti.col[6] = c1.z; ti.col[7] = c1.w;
  } else {
#pragma unroll
    for (int j = 0; j < TL_E; ++j) ti.col[j] = j < cnt ? a.colidx[E0 + le0 + j] : 0;
  }
}

// Folded form (FP32 inner CG): a tile finishes q_v = diag_v p_v - alpha s_v
// of every row that lies inside it, and every tile adds its rows' terms of
// p.q to a per-lane partial: p_v q_v for rows inside, and for a row that
// crosses tiles the linear pieces p_v diag_v p_v (in the tile where it
// starts) and -alpha p_v times the tile's partial (in every tile it touches).
struct Fold {
  const float* diag;
  float alpha;
  float* q;
};

// One tile of s = W x, by one whole warp, from its loaded indices.
template <typename V, bool FOLD = false>
__device__ void tile_finish(const TileArgs<V>& a, const V* __restrict__ x, int64_t t, const TileIn& ti,
                            int32_t* __restrict__ soff, const Fold& fo = Fold{}, float* pq = nullptr) {
  // a row's sum is complete: store it, or (folded) finish q and p.q
  auto put_row = [&](int32_t v, V sv) {
    if (FOLD) {
      const float pv = (float)x[v];
      const float qv = pv * fo.diag[v] - fo.alpha * (float)sv;
      fo.q[v] = qv;
      *pq = fmaf(pv, qv, *pq);
    } else {
      a.s[v] = sv;
    }
  };
  const int lane = threadIdx.x & 31;
  const int64_t E0 = t * TL;
  const int ne = (int)std::min<int64_t>(TL, a.nnz - E0);
  const int32_t rs = ti.rs;
  const uint32_t mw = ti.mw;
  const int le0 = lane * TL_E;
  const int cnt = ne - le0 >= TL_E ? TL_E : (ne - le0 > 0 ? ne - le0 : 0);
  float wt[TL_E];
  if (a.w && a.vec && ne == TL) {
    const float4* w4 = reinterpret_cast<const float4*>(a.w + E0 + le0);
    const float4 w0 = w4[0], w1 = w4[1];
    wt[0] = w0.x; wt[1] = w0.y; wt[2] = w0.z; wt[3] = w0.w;
    wt[4] = w1.x; wt[5] = w1.y; wt[6] = w1.z; wt[7] = w1.w;
  } else {
#pragma unroll
    for (int j = 0; j < TL_E; ++j) wt[j] = j < cnt ? (a.w ? a.w[E0 + le0 + j] : 1.0f) : 0.0f;
  }
  V prod[TL_E];
#pragma unroll
  for (int j = 0; j < TL_E; ++j) prod[j] = j < cnt ? (V)wt[j] * x[ti.col[j]] : (V)0;
  // walk this thread's entries: rf / pf its first row and partial, rl / pl
  // its last; rows that start and end inside the thread are written here
  int32_t rf = 0, rl = INT32_MAX;
  V pf = 0, pl = 0;
  bool ef = false, el = false;
  const bool before = (mw & TM_BEFORE) != 0;
  if (!(mw & TM_GENERAL)) {  // uniform over the tile
    if (cnt > 0) {
      rf = (int32_t)((mw >> TM_RF) & TM_RF_MASK);
      int cur = rf;
      V acc = 0;
      bool first = true;
#pragma unroll
      for (int j = 0; j < TL_E; ++j) {
        if (j < cnt) {
          if (j > 0 && ((mw >> j) & 1u)) {  // entry j starts row cur + 1
            if (first) {
              pf = acc;
              ef = true;
              first = false;
            } else {
              put_row(rs + cur, acc);
            }
            acc = 0;
            ++cur;
          }
          acc += prod[j];
        }
      }
      rl = cur;
      pl = acc;
      el = (mw & TM_EL) != 0;
      if (first) {
        pf = acc;
        ef = el;
      }
    }
  } else {
    const int nr = a.row1[t] - rs + 1;  // rows touching the tile, empty ones included
    const bool use_sm = nr + 1 <= TL_RCAP;
    if (use_sm)
      for (int i = lane; i <= nr; i += TL_T) soff[i] = (int32_t)(a.rowptr[rs + i] - E0);
    __syncwarp();
    auto off = [&](int i) -> int32_t { return use_sm ? soff[i] : (int32_t)(a.rowptr[rs + i] - E0); };
    if (cnt > 0) {
      int lo = 0, hi = nr - 1;  // the row holding entry le0
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off(mid) <= le0) lo = mid;
        else hi = mid - 1;
      }
      rf = lo;
      int cur = lo;
      int32_t beg = off(cur), nxt = off(cur + 1);
      V acc = 0;
      bool first = true;
#pragma unroll
      for (int j = 0; j < TL_E; ++j) {
        if (j < cnt) {
          while (nxt <= le0 + j) {  // row cur ended before this entry
            if (first) {
              pf = acc;
              ef = true;
              first = false;
            } else if (beg < nxt) {
              put_row(rs + cur, acc);
            }
            acc = 0;
            ++cur;
            beg = nxt;
            nxt = off(cur + 1);
          }
          acc += prod[j];
        }
      }
      rl = cur;
      pl = acc;
      el = nxt <= le0 + cnt;
      if (first) {
        pf = acc;
        ef = el;
      }
    }
  }
  // segmented inclusive scan of pl over the lanes, keyed by rl
  V S = pl;
  int32_t key = rl;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const V so = __shfl_up_sync(0xffffffffu, S, d);
    const int32_t ko = __shfl_up_sync(0xffffffffu, key, d);
    if (lane >= d && ko == key) S += so;
  }
  const V Sp = __shfl_up_sync(0xffffffffu, S, 1);  // the previous lane's, for its row
  const int32_t kp = __shfl_up_sync(0xffffffffu, key, 1);
  if (cnt > 0) {
    if (ef) {
      const V tot = (lane > 0 && kp == rf ? Sp : (V)0) + pf;
      if (rf == 0 && before) {
        a.head[t] = tot;
        if (FOLD) *pq = fmaf(-fo.alpha * (float)x[rs], (float)tot, *pq);
      } else {
        put_row(rs + rf, tot);
      }
    }
    if (rl != rf && el) put_row(rs + rl, pl);
    if (le0 + cnt == ne && !el) {  // the tile's last row goes on into the next tile
      if (rl == 0 && before) {
        a.head[t] = S;
        if (FOLD) *pq = fmaf(-fo.alpha * (float)x[rs], (float)S, *pq);
      } else {
        a.tail[t] = S;
        if (FOLD) {
          const int32_t v = rs + rl;
          const float pv = (float)x[v];
          *pq = fmaf(pv, pv * fo.diag[v] - fo.alpha * (float)S, *pq);
        }
      }
    }
  }
  __syncwarp();
}

// The tiles t0, t0 + stride, ... of one warp, each tile's indices loaded
// while the previous tile is summed.
template <typename V, bool FOLD = false>
__device__ __forceinline__ void tile_loop(const TileArgs<V>& a, const V* __restrict__ x, int64_t ntiles, int64_t t0,
                                          int64_t stride, int32_t* __restrict__ soff, const Fold& fo = Fold{},
                                          float* pq = nullptr) {
  TileIn cur, nxt;
  if (t0 < ntiles) tile_load(a, t0, cur);
  for (int64_t t = t0; t < ntiles; t += stride) {
    if (t + stride < ntiles) tile_load(a, t + stride, nxt);
    tile_finish<V, FOLD>(a, x, t, cur, soff, fo, pq);
    cur = nxt;
  }
}

// s_v of a row marked in the span bitmap: 0 if empty, else the sum of its
// tile partials in tile order
template <typename V>
__device__ __forceinline__ V row_total_span(const TileArgs<V>& a, int64_t v) {
  const int64_t e0 = a.rowptr[v], e1 = a.rowptr[v + 1];
  if (e1 <= e0) return (V)0;
  const int64_t t0 = e0 / TL, t1 = (e1 - 1) / TL;
  V s = a.tail[t0];
  for (int64_t t = t0 + 1; t <= t1; ++t) s += a.head[t];
  return s;
}

template <typename V>
__device__ __forceinline__ V row_total(const TileArgs<V>& a, int64_t v) {
  return (a.span[v >> 5] >> (v & 31)) & 1u ? row_total_span(a, v) : a.s[v];
}

// the span bitmap: bit v set when row v is empty or its entries fall in
// more than one tile
__global__ void k_span_bits(int32_t n, const int64_t* __restrict__ rowptr, uint32_t* __restrict__ span,
                            uint32_t* __restrict__ nempty) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool f = false, e = false;
  if (v < n) {
    const int64_t e0 = rowptr[v], e1 = rowptr[v + 1];
    e = e1 <= e0;
    f = e || e0 / TL != (e1 - 1) / TL;
  }
  const uint32_t bits = __ballot_sync(0xffffffffu, f);
  const uint32_t empties = __ballot_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0 && v < n) {
    span[v >> 5] = bits;
    if (empties) atomicAdd(nempty, (uint32_t)__popc(empties));
  }
}

// FP64 s = W x by tiles (the residual of the refinement loop)
__global__ void __launch_bounds__(SV_T) k_tile_rowsum64(TileArgs<double> a, const double* __restrict__ x,
                                                        int64_t ntiles) {
  __shared__ TileSmem sm;
  tile_loop(a, x, ntiles, (int64_t)blockIdx.x * TL_W + (threadIdx.x >> 5), (int64_t)gridDim.x * TL_W,
            sm.off[threadIdx.x >> 5]);
}

// r = b - (sigma + alpha d_w) x + alpha s; partial sums of r.r and b.b
__global__ void __launch_bounds__(SV_T) k_resid_rows(int32_t n, TileArgs<double> a, const double* __restrict__ dw,
                                                     double sigma, double alpha, const double* __restrict__ b,
                                                     const double* __restrict__ x, double* __restrict__ r,
                                                     double* __restrict__ prr, double* __restrict__ pbb) {
  double rr = 0.0, bb = 0.0;
  for (int64_t v = (int64_t)blockIdx.x * SV_T + threadIdx.x; v < n; v += (int64_t)gridDim.x * SV_T) {
    const double ax = x[v] * (sigma + alpha * dw[v]) - alpha * row_total(a, v);
    const double rv = b[v] - ax;
    r[v] = rv;
    rr += rv * rv;
    bb += b[v] * b[v];
  }
  block_sum2(rr, bb);
  if (threadIdx.x == 0) {
    prr[blockIdx.x] = rr;
    pbb[blockIdx.x] = bb;
  }
}

// The whole inner CG in one cooperative launch (one launch per refinement
// step instead of nine per iteration).  An iteration:
//   A  s = W p by tiles                                        | grid barrier
//   B1 q = diag p - alpha s; partials of p.q                   | barrier
//   B2 d += a p, r -= a q, z = r prec; partials of r.z, r.r    | barrier
//   C  p = z + b p                                             | barrier
// Every block sums the partials itself in the same fixed order, so all
// blocks see the same scalars and leave the loop together (the inner
// tolerance rr <= tol2 rr0 is tested every iteration).  FP32 vectors, FP32
// per-thread partials, FP64 sums, as in the per-launch kernels.  The vectors
// start on 16-byte boundaries (B2 and C move four entries per access).
struct CG1 {
  int32_t n;
  int64_t ntiles;
  TileArgs<float> ta;
  const float* diag32;
  const float* prec;  // reciprocal diagonal (Jacobi) or null
  float alpha;
  Inner in;           // r, p, d from k_inner_init; q scratch
  double* part;       // [3][gridDim.x] block partials
  double rz0, rr0, tol2;
  int max_it;
  int* iters_out;
};

// sums of a[0..cnt) and b[0..cnt) in a fixed order (lane-strided, then a
// butterfly in warp 0), valid in every thread of the block; slot[2] is this
// call's own shared scratch (not reused before the next grid barrier)
__device__ __forceinline__ void block_fixed_sum2(const double* a, const double* b, int cnt, double* slot,
                                                 double& sa, double& sb) {
  if (threadIdx.x < 32) {
    double x = 0.0, y = 0.0;
#pragma unroll 4
    for (int i = threadIdx.x; i < cnt; i += 32) {
      x += a[i];
      if (b) y += b[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (threadIdx.x == 0) {
      slot[0] = x;
      slot[1] = y;
    }
  }
  __syncthreads();
  sa = slot[0];
  sb = slot[1];
}

// FOLD (graphs without empty rows): phase A also finishes q and the p.q
// partials, and B1 disappears (three grid barriers per iteration); measured on
// GB300 with 80 registers (3 CTAs per SM; 64 spill): BA 2^20 4.35 -> 4.09 ms
// per solve, 2048^2 grid unchanged (10.7 ms: the tile phase takes longer by
// the per-row loads of p and the diagonal that B1 did in bulk)
template <bool FOLD>
__global__ void __launch_bounds__(SV_T, FOLD ? 3 : 4) k_cg1(CG1 c) {
  cgr::grid_group grid = cgr::this_grid();
  __shared__ TileSmem sm;
  __shared__ double slots[4];
  const int wid = threadIdx.x >> 5;
  const int G = gridDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * SV_T + threadIdx.x;
  const int64_t gstride = (int64_t)G * SV_T;
  const int32_t n = c.n;
  const int64_t n4 = n / 4;
  float4* r4 = reinterpret_cast<float4*>(c.in.r);
  float4* p4 = reinterpret_cast<float4*>(c.in.p);
  float4* d4 = reinterpret_cast<float4*>(c.in.d);
  const float4* q4 = reinterpret_cast<const float4*>(c.in.q);
  const float4* m4 = reinterpret_cast<const float4*>(c.prec);
  const float4* g4 = reinterpret_cast<const float4*>(c.diag32);
  const float4* s4 = reinterpret_cast<const float4*>(c.ta.s);
  float4* q4w = reinterpret_cast<float4*>(c.in.q);
  double rz = c.rz0;
  int it = 0;
  const Fold fo{c.diag32, c.alpha, c.in.q};
  while (it < c.max_it) {
    float pqf = 0.0f;
    if (FOLD) {
      // A: q = diag p - alpha W p for the rows inside a tile, p.q partials
      tile_loop<float, true>(c.ta, c.in.p, c.ntiles, (int64_t)blockIdx.x * TL_W + wid, (int64_t)G * TL_W,
                             sm.off[wid], fo, &pqf);
    } else {
    // A: s = W p
    tile_loop(c.ta, c.in.p, c.ntiles, (int64_t)blockIdx.x * TL_W + wid, (int64_t)G * TL_W, sm.off[wid]);
    grid.sync();
    // B1: q = diag p - alpha s (rows marked in the span bitmap from their
    // tile partials)
    for (int64_t i = gtid; i < n4; i += gstride) {
      const float4 p = p4[i], dg = g4[i];
      float4 sv = s4[i];
      const uint32_t mk = (c.ta.span[i >> 3] >> ((i & 7) * 4)) & 0xFu;
      if (mk) {
        if (mk & 1u) sv.x = row_total_span(c.ta, 4 * i);
        if (mk & 2u) sv.y = row_total_span(c.ta, 4 * i + 1);
        if (mk & 4u) sv.z = row_total_span(c.ta, 4 * i + 2);
        if (mk & 8u) sv.w = row_total_span(c.ta, 4 * i + 3);
      }
      float4 q;
      q.x = p.x * dg.x - c.alpha * sv.x; q.y = p.y * dg.y - c.alpha * sv.y;
      q.z = p.z * dg.z - c.alpha * sv.z; q.w = p.w * dg.w - c.alpha * sv.w;
      q4w[i] = q;
      pqf = fmaf(p.x, q.x, pqf); pqf = fmaf(p.y, q.y, pqf);
      pqf = fmaf(p.z, q.z, pqf); pqf = fmaf(p.w, q.w, pqf);
    }
    for (int64_t v = 4 * n4 + gtid; v < n; v += gstride) {
      const float pv = c.in.p[v];
      const float qv = pv * c.diag32[v] - c.alpha * row_total(c.ta, v);
      c.in.q[v] = qv;
      pqf = fmaf(pv, qv, pqf);
    }
    }
    double pq = pqf, unused = 0.0;
    block_sum2(pq, unused);
    if (threadIdx.x == 0) c.part[blockIdx.x] = pq;
    grid.sync();
    double pq_t, unused2;
    block_fixed_sum2(c.part, nullptr, G, slots, pq_t, unused2);
    const float a = pq_t != 0.0 ? (float)(rz / pq_t) : 0.0f;
    // B2: d += a p, r -= a q
    float rzf = 0.0f, rrf = 0.0f;
    for (int64_t i = gtid; i < n4; i += gstride) {
      const float4 p = p4[i];
      float4 q = q4[i];
      float4 r = r4[i], d = d4[i];
      if (FOLD) {  // rows that cross tiles: q from their tile partials
        const uint32_t mk = (c.ta.span[i >> 3] >> ((i & 7) * 4)) & 0xFu;
        if (mk) {
          const float4 dg = g4[i];
          if (mk & 1u) q.x = p.x * dg.x - c.alpha * row_total_span(c.ta, 4 * i);
          if (mk & 2u) q.y = p.y * dg.y - c.alpha * row_total_span(c.ta, 4 * i + 1);
          if (mk & 4u) q.z = p.z * dg.z - c.alpha * row_total_span(c.ta, 4 * i + 2);
          if (mk & 8u) q.w = p.w * dg.w - c.alpha * row_total_span(c.ta, 4 * i + 3);
        }
      }
      d.x += a * p.x; d.y += a * p.y; d.z += a * p.z; d.w += a * p.w;
      r.x -= a * q.x; r.y -= a * q.y; r.z -= a * q.z; r.w -= a * q.w;
      d4[i] = d;
      r4[i] = r;
      const float4 m = c.prec ? m4[i] : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
      rzf = fmaf(r.x, r.x * m.x, rzf); rzf = fmaf(r.y, r.y * m.y, rzf);
      rzf = fmaf(r.z, r.z * m.z, rzf); rzf = fmaf(r.w, r.w * m.w, rzf);
      rrf = fmaf(r.x, r.x, rrf); rrf = fmaf(r.y, r.y, rrf);
      rrf = fmaf(r.z, r.z, rrf); rrf = fmaf(r.w, r.w, rrf);
    }
    for (int64_t v = 4 * n4 + gtid; v < n; v += gstride) {
      c.in.d[v] += a * c.in.p[v];
      const float qv = FOLD && ((c.ta.span[v >> 5] >> (v & 31)) & 1u)
                           ? c.in.p[v] * c.diag32[v] - c.alpha * row_total_span(c.ta, v)
                           : c.in.q[v];
      const float rv = c.in.r[v] - a * qv;
      c.in.r[v] = rv;
      rzf = fmaf(rv, c.prec ? rv * c.prec[v] : rv, rzf);
      rrf = fmaf(rv, rv, rrf);
    }
    double rzn = rzf, rr = rrf;
    block_sum2(rzn, rr);
    if (threadIdx.x == 0) {
      c.part[G + blockIdx.x] = rzn;
      c.part[2 * G + blockIdx.x] = rr;
    }
    grid.sync();
    double rz_t, rr_t;
    block_fixed_sum2(c.part + G, c.part + 2 * G, G, slots + 2, rz_t, rr_t);
    ++it;
    if (rr_t <= c.tol2 * c.rr0) break;  // the same decision in every block
    // C: p = z + b p
    const float b = rz != 0.0 ? (float)(rz_t / rz) : 0.0f;
    for (int64_t i = gtid; i < n4; i += gstride) {
      const float4 r = r4[i];
      const float4 m = c.prec ? m4[i] : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
      float4 p = p4[i];
      p.x = r.x * m.x + b * p.x; p.y = r.y * m.y + b * p.y;
      p.z = r.z * m.z + b * p.z; p.w = r.w * m.w + b * p.w;
      p4[i] = p;
    }
    for (int64_t v = 4 * n4 + gtid; v < n; v += gstride) {
      const float z = c.prec ? c.in.r[v] * c.prec[v] : c.in.r[v];
      c.in.p[v] = z + b * c.in.p[v];
    }
    rz = rz_t;
    grid.sync();
  }
  if (gtid == 0) *c.iters_out = it;
}

// ---------------------------------------------------------------------------
// Many right-hand sides (m >= 32): the solver's vectors interleaved by
// column, element (v, j) at v m + j.  A warp takes 32 columns of one row, so
// each neighbour gather of the SpMV loads 32 columns' values from one
// contiguous segment (128 bytes in FP32) instead of 32 separate sectors.
// Blocks are 32 x 8 threads (column in the group x row); blockIdx.y is the
// column group and blocks stride over row chunks of 8; per-column partial
// sums go to part[j nb + blockIdx.x] as for the column-major kernels.
// ---------------------------------------------------------------------------
constexpr int IL_R = 8;

__device__ __forceinline__ void il_sum2(double a, double b, int j, bool on, double* __restrict__ pa,
                                        double* __restrict__ pb, int nb) {
  __shared__ double sa[IL_R][33], sb[IL_R][33];
  sa[threadIdx.y][threadIdx.x] = a;
  sb[threadIdx.y][threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.y == 0 && on) {
    double ta = 0.0, tb = 0.0;
    for (int r = 0; r < IL_R; ++r) {
      ta += sa[r][threadIdx.x];
      tb += sb[r][threadIdx.x];
    }
    pa[(size_t)j * nb + blockIdx.x] = ta;
    if (pb) pb[(size_t)j * nb + blockIdx.x] = tb;
  }
}

// [m][n] (column-major) <-> [n][m] (interleaved) through 32 x 32 tiles
__global__ void k_il_transpose(int64_t rows, int64_t cols, const double* __restrict__ src, double* __restrict__ dst) {
  __shared__ double t[32][33];
  for (int64_t br = blockIdx.y; br * 32 < rows; br += gridDim.y)
    for (int64_t bc = blockIdx.x; bc * 32 < cols; bc += gridDim.x) {
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = br * 32 + r, c = bc * 32 + threadIdx.x;
        if (i < rows && c < cols) t[r][threadIdx.x] = src[i * cols + c];
      }
      __syncthreads();
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t c = bc * 32 + r, i = br * 32 + threadIdx.x;
        if (i < rows && c < cols) dst[c * rows + i] = t[threadIdx.x][r];
      }
      __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_resid64_il(int32_t n, int m, const int64_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ colidx, const float* __restrict__ w,
                                                    const double* __restrict__ dw, double sigma, double alpha,
                                                    const double* __restrict__ b, const double* __restrict__ x,
                                                    double* __restrict__ r, double* __restrict__ prr,
                                                    double* __restrict__ pbb, int nb) {
  const int j = blockIdx.y * 32 + threadIdx.x;
  const bool on = j < m;
  double rr = 0.0, bb = 0.0;
  for (int64_t c = blockIdx.x; c * IL_R < n; c += gridDim.x) {
    const int64_t v = c * IL_R + threadIdx.y;
    if (v < n && on) {
      double acc = 0.0;
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
        acc += (w ? (double)w[e] : 1.0) * x[(size_t)colidx[e] * m + j];
      const size_t i = (size_t)v * m + j;
      const double rv = b[i] - (x[i] * (sigma + alpha * dw[v]) - alpha * acc);
      r[i] = rv;
      rr += rv * rv;
      bb += b[i] * b[i];
    }
  }
  il_sum2(rr, bb, j, on, prr, pbb, nb);
}

__global__ void __launch_bounds__(256) k_inner_init_il(int32_t n, int m, const double* __restrict__ r64,
                                                       const float* __restrict__ prec, const double* __restrict__ scal,
                                                       Inner in, double* __restrict__ prz, double* __restrict__ prr,
                                                       int nb) {
  const int j = blockIdx.y * 32 + threadIdx.x;
  const bool on = j < m;
  const double sc = on ? scal[j * 8 + 4] : 0.0;
  float rz = 0.0f, rr = 0.0f;  // per-thread partials in FP32, then FP64 across threads
  for (int64_t c = blockIdx.x; c * IL_R < n; c += gridDim.x) {
    const int64_t v = c * IL_R + threadIdx.y;
    if (v < n && on) {
      const size_t i = (size_t)v * m + j;
      const float rv = (float)(r64[i] * sc);
      const float z = prec ? rv * prec[v] : rv;
      in.r[i] = rv;
      in.p[i] = z;
      in.d[i] = 0.0f;
      rz = fmaf(rv, z, rz);
      rr = fmaf(rv, rv, rr);
    }
  }
  il_sum2(rz, rr, j, on, prz, prr, nb);
}

__global__ void __launch_bounds__(256) k_spmv_pq_il(int32_t n, int m, const int64_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ colidx, const float* __restrict__ w,
                                                    const float* __restrict__ diag32, float alpha, Inner in,
                                                    double* __restrict__ ppq, int nb) {
  const int j = blockIdx.y * 32 + threadIdx.x;
  const bool on = j < m;
  float pq = 0.0f;
  for (int64_t c = blockIdx.x; c * IL_R < n; c += gridDim.x) {
    const int64_t v = c * IL_R + threadIdx.y;
    if (v < n && on) {
      float acc = 0.0f;
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) acc += (w ? w[e] : 1.0f) * in.p[(size_t)colidx[e] * m + j];
      const size_t i = (size_t)v * m + j;
      const float pv = in.p[i];
      const float qv = pv * diag32[v] - alpha * acc;
      in.q[i] = qv;
      pq = fmaf(pv, qv, pq);
    }
  }
  il_sum2(pq, 0.0, j, on, ppq, nullptr, nb);
}

__global__ void __launch_bounds__(256) k_inner_update_il(int32_t n, int m, const float* __restrict__ prec,
                                                         const double* __restrict__ scal, Inner in,
                                                         double* __restrict__ prz, double* __restrict__ prr, int nb) {
  const int j = blockIdx.y * 32 + threadIdx.x;
  const bool on = j < m;
  float a = 0.0f;
  if (on) {
    const double* sc = scal + j * 8;
    a = (sc[5] != 0.0 && sc[1] != 0.0) ? (float)(sc[0] / sc[1]) : 0.0f;
  }
  float rz = 0.0f, rr = 0.0f;
  for (int64_t c = blockIdx.x; c * IL_R < n; c += gridDim.x) {
    const int64_t v = c * IL_R + threadIdx.y;
    if (v < n && on) {
      const size_t i = (size_t)v * m + j;
      in.d[i] += a * in.p[i];
      const float rv = in.r[i] - a * in.q[i];
      in.r[i] = rv;
      const float z = prec ? rv * prec[v] : rv;
      rz = fmaf(rv, z, rz);
      rr = fmaf(rv, rv, rr);
    }
  }
  il_sum2(rz, rr, j, on, prz, prr, nb);
}

__global__ void __launch_bounds__(256) k_inner_p_il(int32_t n, int m, const float* __restrict__ prec,
                                                    const double* __restrict__ scal, Inner in) {
  const int j = blockIdx.y * 32 + threadIdx.x;
  if (j >= m) return;
  const double* sc = scal + j * 8;
  const float beta = sc[0] != 0.0 ? (float)(sc[2] / sc[0]) : 0.0f;
  for (int64_t c = blockIdx.x; c * IL_R < n; c += gridDim.x) {
    const int64_t v = c * IL_R + threadIdx.y;
    if (v < n) {
      const size_t i = (size_t)v * m + j;
      const float z = prec ? in.r[i] * prec[v] : in.r[i];
      in.p[i] = z + beta * in.p[i];
    }
  }
}

__global__ void __launch_bounds__(256) k_correct_il(int32_t n, int m, const double* __restrict__ scal,
                                                    const float* __restrict__ d, double* __restrict__ x) {
  const int j = blockIdx.y * 32 + threadIdx.x;
  if (j >= m) return;
  const double* sc = scal + j * 8;
  if (sc[5] == 0.0) return;
  for (int64_t c = blockIdx.x; c * IL_R < n; c += gridDim.x) {
    const int64_t v = c * IL_R + threadIdx.y;
    if (v < n) {
      const size_t i = (size_t)v * m + j;
      x[i] += (double)d[i] / sc[4];
    }
  }
}

}  // namespace fcx

using namespace fcx;

static fc_status solve_impl(fc_graph* g, int32_t alpha_idx, const double* b, double* x, int32_t n_rhs,
                            double rel_tol, int32_t max_iter, int32_t* iters_out, cudaStream_t st, bool jacobi,
                            double sigma = 1.0) {
  if (g == nullptr || b == nullptr || x == nullptr || n_rhs < 1 || n_rhs > 65535 || alpha_idx < 0 ||
      alpha_idx >= g->n_alpha || !(rel_tol > 0.0) || max_iter < 1) {
    set_error("fc_solve: bad argument");
    return FC_EINVAL;
  }
  const int32_t n = g->n;
  const int m = n_rhs;
  const double alpha = g->alphas[alpha_idx];
  const int nb = (n + SV_T - 1) / SV_T;              // blocks of the element-wise kernels
  const int nbr = (n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;  // blocks of the row kernels
  const size_t nm = (size_t)n * m;
  // many right-hand sides: vectors interleaved by column (see k_spmv_pq_il)
  const bool il = m >= 32;
  const int gy = (m + 31) / 32;
  const int gxi = std::max(1, std::min((n + IL_R - 1) / IL_R, 2048 / gy));
  // scratch: FP64 r64, FP32 r/p/q/d, diag32, partials, scalars
  double* r64 = nullptr;
  float* f32 = nullptr;
  double* part = nullptr;
  double* scal = nullptr;
  // each FP32 vector starts on a 16-byte boundary (four-wide accesses)
  const size_t nmp = (nm + 3) & ~(size_t)3, np4 = ((size_t)n + 3) & ~(size_t)3;
  FC_CK(cudaMallocAsync((void**)&r64, nm * sizeof(double), st));
  FC_CK(cudaMallocAsync((void**)&f32, (4 * nmp + 2 * np4) * sizeof(float), st));
  const int npart = std::max(std::max(nb, nbr), il ? gxi : 1);
  double* bi = nullptr;  // interleaved copies of b and x
  double* xi = nullptr;
  if (il) {
    FC_CK(cudaMallocAsync((void**)&bi, nm * sizeof(double), st));
    FC_CK(cudaMallocAsync((void**)&xi, nm * sizeof(double), st));
    const dim3 tg((unsigned)std::min<int64_t>((n + 31) / 32, 1024), (unsigned)std::min<int64_t>(gy, 1024));
    k_il_transpose<<<tg, dim3(32, 8), 0, st>>>(m, n, b, bi);
    FC_LAUNCHED();
    k_il_transpose<<<tg, dim3(32, 8), 0, st>>>(m, n, x, xi);
    FC_LAUNCHED();
  }
  const double* bv = il ? bi : b;
  double* xv = il ? xi : x;
  const dim3 gridi(gxi, gy), blki(32, IL_R);
  FC_CK(cudaMallocAsync((void**)&part, (size_t)2 * m * npart * sizeof(double) + 4 * m * sizeof(double), st));
  FC_CK(cudaMallocAsync((void**)&scal, (size_t)8 * m * sizeof(double), st));
  Inner in;
  in.r = f32;
  in.p = f32 + nmp;
  in.q = f32 + 2 * nmp;
  in.d = f32 + 3 * nmp;
  in.scal = scal;
  float* diag32 = f32 + 4 * nmp;
  float* inv32 = diag32 + np4;  // the reciprocal of the diagonal
  double* pA = part;
  double* pB = part + (size_t)m * npart;
  double* sums = part + (size_t)2 * m * npart;  // [0..m): rr, [m..2m): bb
  const float* prec = jacobi ? inv32 : nullptr;  // z = r * prec
  k_diag32<<<(n + 255) / 256, 256, 0, st>>>(n, g->dw, sigma, alpha, diag32, inv32);
  FC_LAUNCHED();
  // blocks per column: a few thousand blocks in all, each striding over its
  // column's chunks (many right-hand sides would otherwise launch millions of
  // one-chunk blocks); nbx / nbrx partial sums per column
  const int target = 2048;
  const int nbx = std::max(1, std::min(nb, target / m));
  const int nbrx = std::max(1, std::min(nbr, target / m));
  const dim3 grid(nbx, m);
  const dim3 gridr(nbrx, m);
  const double inner_tol = 1e-4;
  const int check_every = 8;
  // one right-hand side: row sums by edge tiles (FP64 residual and FP32
  // inner products) and the cooperative inner CG (every CTA resident)
  const bool tiles = m == 1;
  const int64_t ntiles = (g->nnz + TL - 1) / TL;
  TileArgs<double> t64{};
  TileArgs<float> t32{};
  void* tile_mem = nullptr;
  int tile_grid = 0;
  bool fold = false;  // q and p.q in the tile phase (graphs without empty rows)
  int cg1_grid = 0;
  double* cg1_part = nullptr;
  if (tiles) {
    const size_t nt = (size_t)std::max<int64_t>(ntiles, 1);
    // [s32 n4][s64 n4][head64 nt][tail64 nt][head32 nt][tail32 nt][row0 nt][row1 nt][meta nt TL_T][span]
    const size_t nsw = ((size_t)n + 31) / 32;
    const size_t bytes = np4 * 12 + nt * 16 + nt * 8 + nt * 8 + nt * TL_T * 4 + nsw * 4 + 16;
    FC_CK(cudaMallocAsync(&tile_mem, bytes, st));
    t32.s = (float*)tile_mem;  // 16-byte aligned: B1 reads it four-wide
    t64.s = (double*)(t32.s + np4);
    t64.head = t64.s + np4;
    t64.tail = t64.head + nt;
    t32.head = (float*)(t64.tail + nt);
    t32.tail = t32.head + nt;
    int32_t* row0 = (int32_t*)(t32.tail + nt);
    int32_t* row1 = row0 + nt;
    uint32_t* meta = (uint32_t*)(row1 + nt);
    uint32_t* span = meta + nt * TL_T;
    uint32_t* nempty = span + nsw;  // rows without entries
    const bool vec = ((uintptr_t)g->colidx % 16 == 0) && (g->w == nullptr || (uintptr_t)g->w % 16 == 0);
    t64.nnz = g->nnz;
    t64.rowptr = g->rowptr;
    t64.colidx = g->colidx;
    t64.w = g->w;
    t64.row0 = row0;
    t64.row1 = row1;
    t64.meta = meta;
    t64.span = span;
    t64.vec = vec;
    t32.nnz = g->nnz;
    t32.rowptr = g->rowptr;
    t32.colidx = g->colidx;
    t32.w = g->w;
    t32.row0 = row0;
    t32.row1 = row1;
    t32.meta = meta;
    t32.span = span;
    t32.vec = vec;
    if (ntiles > 0) {
      k_tile_rows<<<(unsigned)((2 * ntiles + 255) / 256), 256, 0, st>>>(n, g->nnz, g->rowptr, ntiles, row0, row1);
      FC_LAUNCHED();
      k_tile_meta<<<(unsigned)std::min<int64_t>((ntiles + TL_W - 1) / TL_W, 4096), SV_T, 0, st>>>(
          g->nnz, g->rowptr, ntiles, row0, row1, meta);
      FC_LAUNCHED();
    }
    FC_CK(cudaMemsetAsync(nempty, 0, sizeof(uint32_t), st));
    k_span_bits<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, g->rowptr, span, nempty);
    FC_LAUNCHED();
    uint32_t h_nempty = 1;
    FC_CK(cudaMemcpyAsync(&h_nempty, nempty, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    FC_CK(cudaStreamSynchronize(st));
    fold = h_nempty == 0;
    int coop = 0, per_sm = 0, nsm = 0;
    FC_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device));
    FC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device));
    tile_grid = (int)std::max<int64_t>(1, std::min<int64_t>((ntiles + TL_W - 1) / TL_W, (int64_t)8 * nsm));
    FC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fold ? k_cg1<true> : k_cg1<false>, SV_T, 0));
    if (coop && per_sm > 0) {
      cg1_grid = std::min(per_sm, 8) * nsm;
      FC_CK(cudaMallocAsync((void**)&cg1_part, (3 * (size_t)cg1_grid + 1) * sizeof(double), st));
    }
  }
  std::vector<double> h_rr(m), h_bb(m), h_scal((size_t)8 * m, 0.0), h_in(m);
  int used = 0;
  fc_status result = FC_ENOCONV;
  for (int outer = 0; outer < 64; ++outer) {
    int nres = il ? gxi : nbrx;  // residual partials per column
    if (il) {
      k_resid64_il<<<gridi, blki, 0, st>>>(n, m, g->rowptr, g->colidx, g->w, g->dw, sigma, alpha, bv, xv, r64, pA, pB,
                                           gxi);
    } else if (tiles) {
      if (ntiles > 0) {
        k_tile_rowsum64<<<tile_grid, SV_T, 0, st>>>(t64, x, ntiles);
        FC_LAUNCHED();
      }
      k_resid_rows<<<nbx, SV_T, 0, st>>>(n, t64, g->dw, sigma, alpha, b, x, r64, pA, pB);
      nres = nbx;
    } else {
      k_resid64<<<gridr, SV_T, 0, st>>>(n, g->rowptr, g->colidx, g->w, g->dw, sigma, alpha, b, x, r64, pA, pB, nbrx);
    }
    FC_LAUNCHED();
    k_colsum<<<m, SV_T, 0, st>>>(pA, nres, sums);
    fcx::note_launch();
    k_colsum<<<m, SV_T, 0, st>>>(pB, nres, sums + m);
    fcx::note_launch();
    if (sigma == 0.0) {  // singular L: keep the residual in L's range
      k_proj_mean<<<m, SV_T, 0, st>>>(n, m, il, r64, sums);
      FC_LAUNCHED();
    }
    FC_CK(cudaMemcpyAsync(h_rr.data(), sums, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    FC_CK(cudaMemcpyAsync(h_bb.data(), sums + m, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    FC_CK(cudaStreamSynchronize(st));
    bool all_ok = true;
    for (int j = 0; j < m; ++j) {
      const double rn = std::sqrt(h_rr[j]), bn = std::sqrt(h_bb[j]);
      const bool ok = rn <= rel_tol * bn || rn == 0.0;
      h_scal[(size_t)j * 8 + 5] = ok ? 0.0 : 1.0;
      h_scal[(size_t)j * 8 + 4] = rn > 0.0 ? 1.0 / rn : 1.0;
      all_ok = all_ok && ok;
    }
    if (all_ok) {
      result = FC_OK;
      break;
    }
    if (used >= max_iter) break;
    FC_CK(cudaMemcpyAsync(scal, h_scal.data(), (size_t)8 * m * sizeof(double), cudaMemcpyHostToDevice, st));
    if (il)
      k_inner_init_il<<<gridi, blki, 0, st>>>(n, m, r64, prec, scal, in, pA, pB, gxi);
    else
      k_inner_init<<<grid, SV_T, 0, st>>>(n, r64, prec, scal, in, pA, pB, nbx);
    FC_LAUNCHED();
    k_colsum<<<m, SV_T, 0, st>>>(pA, il ? gxi : nbx, sums);
    fcx::note_launch();
    k_colsum<<<m, SV_T, 0, st>>>(pB, il ? gxi : nbx, sums + m);
    fcx::note_launch();
    FC_CK(cudaMemcpyAsync(h_in.data(), sums, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    FC_CK(cudaMemcpyAsync(h_rr.data(), sums + m, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    FC_CK(cudaStreamSynchronize(st));
    std::vector<double> rr0(h_rr);
    for (int j = 0; j < m; ++j) h_scal[(size_t)j * 8 + 0] = h_in[j];
    FC_CK(cudaMemcpyAsync(scal, h_scal.data(), (size_t)8 * m * sizeof(double), cudaMemcpyHostToDevice, st));
    if (cg1_grid > 0) {
      // one right-hand side: the inner CG in one cooperative launch
      CG1 c;
      c.n = n;
      c.ntiles = ntiles;
      c.ta = t32;
      c.diag32 = diag32;
      c.prec = prec;
      c.alpha = (float)alpha;
      c.in = in;
      c.part = cg1_part;
      c.rz0 = h_in[0];
      c.rr0 = rr0[0];
      c.tol2 = inner_tol * inner_tol;
      c.max_it = max_iter - used;
      c.iters_out = (int*)(cg1_part + 3 * cg1_grid);
      void* args[] = {&c};
      FC_CK(cudaLaunchCooperativeKernel(fold ? (void*)k_cg1<true> : (void*)k_cg1<false>, dim3(cg1_grid),
                                        dim3(SV_T), args, 0, st));
      FC_LAUNCHED();
      int done = 0;
      FC_CK(cudaMemcpyAsync(&done, c.iters_out, sizeof(int), cudaMemcpyDeviceToHost, st));
      FC_CK(cudaStreamSynchronize(st));
      used += done;
    }
    int it = 0;
    while (cg1_grid == 0 && used < max_iter) {
      if (il)
        k_spmv_pq_il<<<gridi, blki, 0, st>>>(n, m, g->rowptr, g->colidx, g->w, diag32, (float)alpha, in, pA, gxi);
      else
        k_spmv_pq<<<gridr, SV_T, 0, st>>>(n, g->rowptr, g->colidx, g->w, diag32, (float)alpha, in, pA, nbrx);
      FC_LAUNCHED();
      // pq -> scal[j*8+1]
      k_colsum<<<m, SV_T, 0, st>>>(pA, il ? gxi : nbrx, sums);
      fcx::note_launch();
      k_put_scal<<<(m + 127) / 128, 128, 0, st>>>(m, sums, 1, 1, scal);
      FC_LAUNCHED();
      if (il)
        k_inner_update_il<<<gridi, blki, 0, st>>>(n, m, prec, scal, in, pA, pB, gxi);
      else
        k_inner_update<<<grid, SV_T, 0, st>>>(n, prec, scal, in, pA, pB, nbx);
      FC_LAUNCHED();
      k_colsum<<<m, SV_T, 0, st>>>(pA, il ? gxi : nbx, sums);
      fcx::note_launch();
      k_colsum<<<m, SV_T, 0, st>>>(pB, il ? gxi : nbx, sums + m);
      fcx::note_launch();
      k_put_scal<<<(m + 127) / 128, 128, 0, st>>>(m, sums, 2, 2, scal);  // scal[2] <- sums[0..m), scal[3] <- sums[m..2m)
      FC_LAUNCHED();
      if (il)
        k_inner_p_il<<<gridi, blki, 0, st>>>(n, m, prec, scal, in);
      else
        k_inner_p<<<grid, SV_T, 0, st>>>(n, prec, scal, in);
      FC_LAUNCHED();
      k_scal_shift<<<(m + 127) / 128, 128, 0, st>>>(m, scal);
      fcx::note_launch();
      ++used;
      ++it;
      if (it == 1 || it == 2 || it == 4 || it % check_every == 0) {
        FC_CK(cudaMemcpyAsync(h_rr.data(), sums + m, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        FC_CK(cudaStreamSynchronize(st));
        bool conv = true;
        for (int j = 0; j < m; ++j)
          if (h_scal[(size_t)j * 8 + 5] != 0.0 && std::sqrt(h_rr[j]) > inner_tol * std::sqrt(rr0[j])) conv = false;
        if (conv) break;
      }
    }
    if (il)
      k_correct_il<<<gridi, blki, 0, st>>>(n, m, scal, in.d, xv);
    else
      k_correct<<<grid, SV_T, 0, st>>>(n, scal, in.d, x);
    FC_LAUNCHED();
  }
  if (il) {
    const dim3 tg((unsigned)std::min<int64_t>(gy, 1024), (unsigned)std::min<int64_t>((n + 31) / 32, 1024));
    k_il_transpose<<<tg, dim3(32, 8), 0, st>>>(n, m, xi, x);
    FC_LAUNCHED();
    FC_CK(cudaFreeAsync(bi, st));
    FC_CK(cudaFreeAsync(xi, st));
  }
  FC_CK(cudaFreeAsync(r64, st));
  FC_CK(cudaFreeAsync(f32, st));
  FC_CK(cudaFreeAsync(part, st));
  FC_CK(cudaFreeAsync(scal, st));
  if (cg1_part) FC_CK(cudaFreeAsync(cg1_part, st));
  if (tile_mem) FC_CK(cudaFreeAsync(tile_mem, st));
  FC_CK(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = used;
  if (result != FC_OK) set_error("fc_solve: max_iter reached before rel_tol");
  return result;
}

extern "C" fc_status fc_solve(fc_graph* g, int32_t alpha_idx, const double* b, double* x, int32_t n_rhs,
                              double rel_tol, int32_t max_iter, int32_t* iters_out, void* stream) {
  return solve_impl(g, alpha_idx, b, x, n_rhs, rel_tol, max_iter, iters_out, (cudaStream_t)stream, true);
}

extern "C" fc_status fc_pivot_solve(fc_graph* g, int32_t alpha_idx, double* x, double rel_tol, int32_t max_iter,
                                    int32_t* iters_out, void* stream) {
  if (g == nullptr || x == nullptr || alpha_idx < 0 || alpha_idx >= g->n_alpha) {
    set_error("fc_pivot_solve: bad argument");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  double* rhs = nullptr;
  double* part = nullptr;
  const int64_t n1 = (int64_t)n + 1;
  const int nb = (int)((n1 + SV_T - 1) / SV_T);
  FC_CK(cudaMallocAsync((void**)&rhs, (size_t)n * sizeof(double), st));
  FC_CK(cudaMallocAsync((void**)&part, (size_t)(nb + 1) * sizeof(double), st));
  // grounded system: x(u*) = 0, (I + alpha L) x_V = -1/(n+1) 1
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, -1.0 / (double)n1, rhs);
  FC_LAUNCHED();
  FC_CK(cudaMemsetAsync(x, 0, (size_t)n1 * sizeof(double), st));
  // The right-hand side restricted to V is a multiple of 1, an eigenvector of
  // I + alpha L with eigenvalue 1: unpreconditioned CG reaches it in one step
  // (Jacobi scaling would break that), so the pivot system runs without it.
  const fc_status s = solve_impl(g, alpha_idx, rhs, x, 1, rel_tol, max_iter, iters_out, st, false);
  if (s != FC_OK && s != FC_ENOCONV) return s;
  // shift to the mean-zero gauge of L*^+
  k_partial_sum<<<nb, SV_T, 0, st>>>(n1, x, part);
  fcx::note_launch();
  k_colsum<<<1, SV_T, 0, st>>>(part, nb, part + nb);
  fcx::note_launch();
  k_shift<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(n1, part + nb, x);
  FC_LAUNCHED();
  FC_CK(cudaFreeAsync(rhs, st));
  FC_CK(cudaFreeAsync(part, st));
  FC_CK(cudaStreamSynchronize(st));
  return s;
}

// Column sums of an [m][n] block (one block per column, fixed order) and the
// mean of each column subtracted: out[j][v] = in[j][v] - sum_j / n.
__global__ void k_col_mean_sub(int32_t n, const double* __restrict__ in, double* __restrict__ out) {
  __shared__ double red[SV_T];
  const size_t off = (size_t)blockIdx.x * n;
  double s = 0.0;
  for (int64_t v = threadIdx.x; v < n; v += SV_T) s += in[off + v];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = SV_T / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  const double mean = red[0] / (double)n;
  for (int64_t v = threadIdx.x; v < n; v += SV_T) out[off + v] = in[off + v] - mean;
}

extern "C" fc_status fc_laplacian_solve(fc_graph* g, const double* b, double* x, int32_t n_rhs, double rel_tol,
                                        int32_t max_iter, int32_t* iters_out, void* stream) {
  if (g == nullptr || b == nullptr || x == nullptr || n_rhs < 1 || n_rhs > 65535) {
    set_error("fc_laplacian_solve: bad argument");
    return FC_EINVAL;
  }
  if (g->root < 0) {
    set_error("fc_laplacian_solve: needs a graph from fc_build_rooted (G connected)");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  double* rhs = nullptr;
  FC_CK(cudaMallocAsync((void**)&rhs, (size_t)n * n_rhs * sizeof(double), st));
  // b projected onto the range of L (the complement of span(1))
  k_col_mean_sub<<<n_rhs, SV_T, 0, st>>>(n, b, rhs);
  FC_LAUNCHED();
  const fc_status s = solve_impl(g, 0, rhs, x, n_rhs, rel_tol, max_iter, iters_out, st, true, 0.0);
  if (s == FC_OK || s == FC_ENOCONV) {
    // the mean-zero solution: L^+ b
    k_col_mean_sub<<<n_rhs, SV_T, 0, st>>>(n, x, x);
    FC_LAUNCHED();
  }
  FC_CK(cudaFreeAsync(rhs, st));
  FC_CK(cudaStreamSynchronize(st));
  return s;
}
