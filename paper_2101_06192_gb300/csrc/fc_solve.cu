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
#include <algorithm>
#include <cmath>
#include <vector>

#include "fc_internal.cuh"

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
  FC_CK(cudaMallocAsync((void**)&r64, nm * sizeof(double), st));
  FC_CK(cudaMallocAsync((void**)&f32, (4 * nm + 2 * (size_t)n) * sizeof(float), st));
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
  in.p = f32 + nm;
  in.q = f32 + 2 * nm;
  in.d = f32 + 3 * nm;
  in.scal = scal;
  float* diag32 = f32 + 4 * nm;
  float* inv32 = diag32 + n;  // the reciprocal of the diagonal
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
  std::vector<double> h_rr(m), h_bb(m), h_scal((size_t)8 * m, 0.0), h_in(m);
  int used = 0;
  fc_status result = FC_ENOCONV;
  for (int outer = 0; outer < 64; ++outer) {
    if (il)
      k_resid64_il<<<gridi, blki, 0, st>>>(n, m, g->rowptr, g->colidx, g->w, g->dw, sigma, alpha, bv, xv, r64, pA, pB,
                                           gxi);
    else
      k_resid64<<<gridr, SV_T, 0, st>>>(n, g->rowptr, g->colidx, g->w, g->dw, sigma, alpha, b, x, r64, pA, pB, nbrx);
    FC_LAUNCHED();
    k_colsum<<<m, SV_T, 0, st>>>(pA, il ? gxi : nbrx, sums);
    fcx::note_launch();
    k_colsum<<<m, SV_T, 0, st>>>(pB, il ? gxi : nbrx, sums + m);
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
    int it = 0;
    while (used < max_iter) {
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
