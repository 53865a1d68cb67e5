// Group forest closeness (Sec. 5, Algorithm 3): the greedy maximiser of
// 1 / tr((L*_{-S})^{-1}) over groups S of k vertices.
//
// Algorithm 3 starts from the vertex v0 of highest individual forest
// closeness, keeps M = (L*_{-S})^{-1} and at every step adds the vertex v of
// V \ S (never u*) with the largest gain ||M e_v||^2 / M_vv, then applies the
// rank-one downdate M - (M e_v)(M e_v)^T / M_vv and drops v's row and column.
//
// GB300 design:
//  * The starting inverse.  The paper takes a dense pseudo-inverse of L* and
//    a dense inverse of L*_{-v0}.  Here the forest matrix Omega = (I +
//    alpha L)^{-1} is solved column by column with the library's FP64-refined
//    CG (I + alpha L is sparse and well conditioned; a dense O(n^3) FP64
//    factorisation would run on GB300's small FP64 rate), v0 = argmin
//    Omega_vv (the order of n L*^+[v, v] + tr L*^+), and
//        (L*_{-v0})^{-1}[a, b] = Omega_ab - Omega_a,v0 - Omega_v0,b + Omega_v0,v0
//    with Omega's u* row and column read as zero (grounding at v0 instead of
//    u*; both sides are the same Green's function of G*).
//  * The greedy.  M is kept as a dense (n+1) x (n+1) FP64 matrix (index n =
//    u*); a chosen vertex's row and column become zero instead of being
//    removed.  One fused pass per step applies the downdate to every row and
//    accumulates the new row's squared norm and diagonal (M is symmetric, so
//    row norms are the column norms of the gain), the gain of every
//    candidate; a one-block kernel takes the argmax (ties: smallest id).  The
//    pass streams M once (read + write, 16 bytes per entry) and does two FP64
//    FMAs per entry; everything stays on the device, with no host
//    synchronisation inside the loop.
#include <algorithm>
#include <cfloat>

#include "fc_internal.cuh"

namespace fcx {

namespace {

constexpr int GR_T = 256;

// Identity block: B[c][r] = (r == j0 + c), c in [0, nb), r in [0, n).
__global__ void k_grp_eye(int32_t n, int32_t j0, int32_t nb, double* __restrict__ B) {
  const int64_t tot = (int64_t)n * nb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / n, r = i - c * n;
    B[i] = (r == j0 + c) ? 1.0 : 0.0;
  }
}

// v0 = argmin_v Omega_vv, ties to the smallest id (one block).
__global__ void k_grp_first(int32_t n, const double* __restrict__ Om, int32_t* __restrict__ v_out,
                            int32_t* __restrict__ S0, uint8_t* __restrict__ chosen) {
  __shared__ double sb[GR_T];
  __shared__ int32_t si[GR_T];
  double best = DBL_MAX;
  int32_t bi = 0x7fffffff;
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const double d = Om[(int64_t)v * n + v];
    if (d < best || (d == best && v < bi)) {
      best = d;
      bi = v;
    }
  }
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sb[threadIdx.x + s];
      const int32_t oi = si[threadIdx.x + s];
      if (o < sb[threadIdx.x] || (o == sb[threadIdx.x] && oi < si[threadIdx.x])) {
        sb[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *v_out = si[0];
    S0[0] = si[0];
    chosen[si[0]] = 1;
  }
}

// M[a][b] for a, b in [0, n] (n = u*) from Omega (row-major, Omega_ab =
// Om[a n + b]), grounded at v0; v0's row and column are zero.
__global__ void k_grp_form(int32_t n, int64_t ld, const double* __restrict__ Om, const int32_t* __restrict__ vp,
                           double* __restrict__ M) {
  const int32_t v0 = *vp;
  const int32_t n1 = n + 1;
  const double dvv = Om[(int64_t)v0 * n + v0];
  for (int64_t a = blockIdx.x; a < n1; a += gridDim.x) {
    const double oav = a < n ? Om[a * n + v0] : 0.0;
    double* row = M + a * ld;
    for (int32_t b = threadIdx.x; b < n1; b += blockDim.x) {
      double val = 0.0;
      if (a != v0 && b != v0) {
        const double oab = (a < n && b < n) ? Om[a * n + b] : 0.0;
        const double ovb = b < n ? Om[(int64_t)v0 * n + b] : 0.0;
        val = oab - oav - ovb + dvv;
      }
      row[b] = val;
    }
  }
}

// One greedy step's pass over the rows.  With v >= 0 the row a becomes
// M_a - (m_a / m_v) m (m = the saved row v), exactly zero in row v and
// column v; with v < 0 the rows are only read.  Each row's squared norm and
// diagonal give gain[a] = norm / diag for candidates (a < n, not chosen),
// -1 otherwise; diag[a] receives the new diagonal entry.
__global__ void __launch_bounds__(GR_T) k_grp_pass(int32_t n, int64_t ld, double* __restrict__ M,
                                                   const double* __restrict__ m, const int32_t* __restrict__ vp,
                                                   const uint8_t* __restrict__ chosen, double* __restrict__ gain,
                                                   double* __restrict__ diag) {
  __shared__ double red[GR_T / 32];
  const int32_t n1 = n + 1;
  const int32_t v = vp ? *vp : -1;
  const double mv = v >= 0 ? m[v] : 1.0;
  for (int64_t a = blockIdx.x; a < n1; a += gridDim.x) {
    double* row = M + a * ld;
    double ss = 0.0;
    if (v >= 0 && a == v) {
      for (int32_t b = threadIdx.x; b < n1; b += blockDim.x) row[b] = 0.0;
    } else if (v >= 0) {
      const double c = m[a] / mv;
      for (int32_t b = threadIdx.x; b < n1; b += blockDim.x) {
        const double x = b == v ? 0.0 : fma(-c, m[b], row[b]);
        row[b] = x;
        ss = fma(x, x, ss);
      }
    } else {
      for (int32_t b = threadIdx.x; b < n1; b += blockDim.x) {
        const double x = row[b];
        ss = fma(x, x, ss);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();  // also makes this block's writes of the row visible to thread 0
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < GR_T / 32; ++w) t += red[w];
      const double d = row[a];
      diag[a] = d;
      gain[a] = (a < n && !chosen[a] && d > 0.0) ? t / d : -1.0;
    }
    __syncthreads();
  }
}

// argmax of gain (ties: smallest id), one block; records the choice, marks
// it chosen and saves its row (the column, by symmetry) for the next pass.
__global__ void k_grp_pick(int32_t n, int64_t ld, const double* __restrict__ gain, const double* __restrict__ M,
                           int32_t step, int32_t* __restrict__ vp, int32_t* __restrict__ S, uint8_t* __restrict__ chosen,
                           double* __restrict__ m) {
  __shared__ double sb[GR_T];
  __shared__ int32_t si[GR_T];
  double best = -DBL_MAX;
  int32_t bi = 0x7fffffff;
  for (int32_t a = threadIdx.x; a < n; a += blockDim.x) {
    const double x = gain[a];
    if (x > best || (x == best && a < bi)) {
      best = x;
      bi = a;
    }
  }
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sb[threadIdx.x + s];
      const int32_t oi = si[threadIdx.x + s];
      if (o > sb[threadIdx.x] || (o == sb[threadIdx.x] && oi < si[threadIdx.x])) {
        sb[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int32_t v = si[0];
  if (threadIdx.x == 0) {
    *vp = v;
    S[step] = v;
    chosen[v] = 1;
  }
  for (int32_t b = threadIdx.x; b <= n; b += blockDim.x) m[b] = M[(int64_t)v * ld + b];
}

// farness[step] = sum of the diagonal (one block; fixed order per thread,
// then a fixed tree).
__global__ void k_grp_trace(int32_t n, const double* __restrict__ diag, int32_t step, double* __restrict__ far) {
  __shared__ double sb[GR_T];
  double t = 0.0;
  for (int32_t a = threadIdx.x; a <= n; a += blockDim.x) t += diag[a];
  sb[threadIdx.x] = t;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sb[threadIdx.x] += sb[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) far[step] = sb[0];
}

}  // namespace

}  // namespace fcx

using namespace fcx;

extern "C" fc_status fc_group_closeness(fc_graph* g, int32_t alpha_idx, int32_t k, double rel_tol, int32_t* S_out,
                                        double* farness_out, void* stream) {
  if (g == nullptr || S_out == nullptr || alpha_idx < 0 || alpha_idx >= g->n_alpha || k < 1 || k > g->n ||
      !(rel_tol > 0.0) || g->num_graphs > 0) {
    set_error("fc_group_closeness: bad argument (single graphs only, 1 <= k <= n)");
    return FC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  const int32_t n1 = n + 1;
  const int64_t ld = ((int64_t)n1 + 3) & ~(int64_t)3;  // row stride of M: 32-byte aligned rows
  int nsm = 0;
  FC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device));
  // Omega (n^2), M (n1 x ld), the identity block and the solver's scratch
  // (FP64 residual, four FP32 vectors and, for 32 or more right-hand sides,
  // interleaved copies of b and x: about 40 bytes per right-hand side and vertex)
  const int32_t nb = std::min<int32_t>(n, 4096);
  const size_t need = (size_t)n * n * 8 + (size_t)n1 * ld * 8 + (size_t)nb * n * (8 + 40);
  size_t freeb = 0, totb = 0;
  FC_CK(cudaMemGetInfo(&freeb, &totb));
  if (need > freeb / 10 * 9) {
    set_error("fc_group_closeness: the dense matrices do not fit in device memory");
    return FC_ENOMEM;
  }
  double *Om = nullptr, *M = nullptr, *B = nullptr, *vec = nullptr;
  int32_t* vp = nullptr;
  uint8_t* chosen = nullptr;
  FC_CK(cudaMallocAsync((void**)&Om, (size_t)n * n * 8, st));
  FC_CK(cudaMallocAsync((void**)&B, (size_t)nb * n * 8, st));
  // Omega, column block by column block (column j is also row j: symmetric)
  fc_status r = FC_OK;
  for (int32_t j0 = 0; j0 < n && r == FC_OK; j0 += nb) {
    const int32_t cnt = std::min(nb, n - j0);
    const unsigned eb = (unsigned)std::min<int64_t>(((int64_t)cnt * n + GR_T - 1) / GR_T, (int64_t)nsm * 16);
    k_grp_eye<<<eb, GR_T, 0, st>>>(n, j0, cnt, B);
    FC_LAUNCHED();
    double* X = Om + (size_t)j0 * n;
    FC_CK(cudaMemsetAsync(X, 0, (size_t)cnt * n * 8, st));
    r = fc_solve(g, alpha_idx, B, X, cnt, rel_tol, 100000, nullptr, stream);
  }
  FC_CK(cudaFreeAsync(B, st));
  if (r != FC_OK) {
    FC_CK(cudaFreeAsync(Om, st));
    return r;
  }
  FC_CK(cudaMallocAsync((void**)&M, (size_t)n1 * ld * 8, st));
  FC_CK(cudaMallocAsync((void**)&vec, (size_t)3 * ld * 8, st));  // m, gain, diag
  FC_CK(cudaMallocAsync((void**)&vp, 16, st));
  FC_CK(cudaMallocAsync((void**)&chosen, (size_t)n1, st));
  double* m = vec;
  double* gain = vec + ld;
  double* diag = vec + 2 * ld;
  FC_CK(cudaMemsetAsync(chosen, 0, (size_t)n1, st));
  k_grp_first<<<1, GR_T, 0, st>>>(n, Om, vp, S_out, chosen);
  FC_LAUNCHED();
  const unsigned rb = (unsigned)std::min<int64_t>(n1, (int64_t)nsm * 8);
  k_grp_form<<<rb, GR_T, 0, st>>>(n, ld, Om, vp, M);
  FC_LAUNCHED();
  FC_CK(cudaFreeAsync(Om, st));
  // gains of the starting inverse; v0's row is zero, so its gain is -1
  k_grp_pass<<<rb, GR_T, 0, st>>>(n, ld, M, m, nullptr, chosen, gain, diag);
  FC_LAUNCHED();
  if (farness_out) {
    k_grp_trace<<<1, GR_T, 0, st>>>(n, diag, 0, farness_out);
    FC_LAUNCHED();
  }
  for (int32_t step = 1; step < k; ++step) {
    k_grp_pick<<<1, GR_T, 0, st>>>(n, ld, gain, M, step, vp, S_out, chosen, m);
    FC_LAUNCHED();
    k_grp_pass<<<rb, GR_T, 0, st>>>(n, ld, M, m, vp, chosen, gain, diag);
    FC_LAUNCHED();
    if (farness_out) {
      k_grp_trace<<<1, GR_T, 0, st>>>(n, diag, step, farness_out);
      FC_LAUNCHED();
    }
  }
  FC_CK(cudaFreeAsync(M, st));
  FC_CK(cudaFreeAsync(vec, st));
  FC_CK(cudaFreeAsync(vp, st));
  FC_CK(cudaFreeAsync(chosen, st));
  FC_CK(cudaStreamSynchronize(st));
  return FC_OK;
}
