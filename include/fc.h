/*
 * fc -- forest closeness on GB300 (sm_103a): C ABI.
 *
 * Estimates diag(Omega), Omega = (I + alpha L)^{-1}, the forest farness and the
 * forest closeness of every vertex of a simple undirected graph by sampling
 * uniform spanning trees of the augmented graph G* with Wilson's algorithm, as
 * in van der Grinten, Angriman, Predari, Meyerhenke, "New Approximation
 * Algorithms for Forest Closeness Centrality" (arXiv 2101.06192):
 *   forest matrix / distance / closeness    Sec. 2, Def. 1, Def. 2
 *   augmented graph G*, pivot u*            Sec. 4.1, Prop. 2
 *   estimator and its parameters            Algorithm 1, Prop. 1, Thm. 1 (Sec. 4.2)
 *   tree sampler                            Algorithm 2 (App. B)
 *   farness from the diagonal               Eq. 3
 *
 * Conventions (all entry points):
 *   - Graphs are CSR: rowptr int64[n+1], colidx int32[nnz], optional weights
 *     float32[nnz].  Rows sorted ascending, no self-loops, no duplicates,
 *     symmetric (with equal weights both ways), weights finite and >= 0
 *     (Sec. 2: finite simple undirected graphs with non-negative weights).
 *   - The universal vertex u* has index n.
 *   - Unless a flag says otherwise every pointer argument is a DEVICE pointer
 *     owned by the caller; the library never frees caller memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; calls that report device-side errors synchronise the
 *     stream before returning, as stated per function.
 *   - No function throws; every failure is a status code.  On failure the
 *     outputs are unspecified unless stated otherwise.
 *   - fc_graph is not thread-safe: use one graph per host thread or serialise.
 */
#ifndef FC_H_
#define FC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc_graph fc_graph;

typedef enum {
  FC_OK = 0,
  FC_EINVAL = 1,     /* bad argument or input graph violates the CSR contract */
  FC_ENOMEM = 2,     /* device or host allocation failed                      */
  FC_ECUDA = 3,      /* a CUDA runtime call failed                            */
  FC_ENOCONV = 4,    /* solver hit max_iter before rel_tol (best x written)   */
  FC_ETIMEOUT = 5,   /* sampler watchdog: iteration budget exhausted          */
  FC_EOVERFLOW = 6   /* a per-vertex visit counter exceeded 2^24 - 1          */
} fc_status;

/* flags for fc_build_augmented */
#define FC_HOST_PTRS 0u   /* rowptr/colidx/w/alphas are host pointers   */
#define FC_DEVICE_PTRS 1u /* rowptr/colidx/w are device pointers (alphas: host) */

/*
 * Build G* (Sec. 4.1; first step of Algorithm 1) for n_alpha values of alpha
 * over one CSR graph G.  Copies the CSR into memory owned by the returned graph
 * and derives, on the device: degrees, weighted degrees d_w (FP64, summed left
 * to right per row), the per-row FP64 prefix sums of the weights, the
 * ascending-degree start order of Algorithm 2 (ties by vertex id), and, per
 * alpha, the integer selection thresholds of the random-stack selector.
 * Selector (one stack entry of v with degree d, Philox words o0..o3):
 *   u53 = (o0 << 21) | (o1 >> 11);  U = u53 * 2^-53;
 *   unweighted: t = fl(1 + fl(alpha d)); x = fl(U t), clamped to the largest
 *     double below t; x < 1 selects u*, else neighbour floor(o2 d / 2^32);
 *   weighted: t_0 = 1, t_j = fl(1 + fl(alpha S_j)) with S_j the FP64 prefix of
 *     the row's weights; x = fl(U t_d) clamped below t_d; slot = first j with
 *     x < t_j (slot 0 = u*, slot j = j-th neighbour).
 * The thresholds are the exact integer boundaries of these FP64 comparisons,
 * so the walk itself compares integers only.
 *   n >= 1 and n < 2^30; 0 <= nnz < 2^32; 1 <= n_alpha <= 64;
 *   alphas[i] finite and > 0 (alphas is always a host pointer);
 *   w == NULL means unweighted (every edge weight 1).
 * Validates the CSR contract above on the device; FC_EINVAL if violated.
 * Synchronises `stream`.  On success *out owns device memory until fc_destroy.
 */
fc_status fc_build_augmented(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                             const float* w, const double* alphas, int32_t n_alpha, uint32_t flags,
                             void* stream, fc_graph** out);

/*
 * A batch of graphs sampled together (one persistent launch): the graphs are
 * given as one block-diagonal CSR over n = vertex_offsets[num_graphs] vertices
 * (graph i owns vertices [vertex_offsets[i], vertex_offsets[i+1]); no edge may
 * leave its graph -- FC_EINVAL otherwise), each with its own alpha
 * (graph_alphas[i], host).  vertex_offsets is a host array of num_graphs + 1
 * entries starting at 0, every graph non-empty.  Because G* of the union is
 * the union of the graphs' G* glued at u*, a spanning tree of it is one tree
 * per graph, and all the per-vertex entry points below apply unchanged with
 * vertex ids of the union, alpha index 0:
 *   fc_sample_usts   samples tau trees of every graph: work items (graph,
 *                    tree) run largest graph first; steps_out is [graph][tree];
 *                    parents is [tree][n]; the random stacks use union vertex
 *                    ids, so results equal those of the union graph.
 *   fc_forest_farness  Eq. 3 and Def. 2 within each graph (its n and trace).
 *   fc_batch_latency   per-graph completion time of the last launch.
 * Other arguments as fc_build_augmented.  Synchronises `stream`.
 */
fc_status fc_build_batch(int32_t num_graphs, const int64_t* vertex_offsets, int64_t nnz, const int64_t* rowptr,
                         const int32_t* colidx, const float* w, const double* graph_alphas, uint32_t flags,
                         void* stream, fc_graph** out);

/*
 * Per-graph latency of the last fc_sample_usts on a batch graph: for graph i,
 * the time from the first CTA start of the launch to the completion of the
 * graph's last tree, in ms (%globaltimer).  per_graph_ms: host double[G].
 * Synchronous.
 */
fc_status fc_batch_latency(fc_graph* g, double* per_graph_ms);

/* Graph metadata (host pointers; any may be NULL). */
fc_status fc_graph_info(const fc_graph* g, int32_t* n, int64_t* nnz, int32_t* n_alpha,
                        int32_t* weighted);

/*
 * Sampler launch shape.  walkers_per_tree: concurrent Wilson walkers sharing
 * one tree (a multiple of 32 in [32, 1024], 0 = automatic); max_trees_resident:
 * cap on trees in flight (0 = fill the GPU); smem: 0 = automatic, 1 = force
 * global-memory tree state, 2 = force shared-memory tree state (FC_EINVAL if
 * it does not fit); regs: register cap of the kernel variant (32, 40, 48 or
 * 64; 0 = automatic; the CSR-walk kernel maps 48 to 40, the edge-record kernel
 * maps 32 to 40).  Affects speed only, never results.
 */
fc_status fc_set_sampler_shape(fc_graph* g, int32_t walkers_per_tree, int32_t max_trees_resident,
                               int32_t smem, int32_t regs);

/*
 * Order in which the sampler's walkers take start vertices: 0 = ascending
 * degree (Algorithm 2's order), 1 = descending degree, 2 = ascending vertex
 * id, 3 = descending vertex id, 4 = automatic (the default: ascending vertex id
 * unless more than a quarter of the CSR entries join vertices at most 32 ids
 * apart, then ascending degree).  The trees do not depend on it (cycle
 * popping); only the amount of waiting between concurrent walkers and the
 * locality of the first steps do (vertex-id order loads start windows
 * coalesced but makes walkers collide on graphs whose ids follow geometry).
 */
fc_status fc_set_start_order(fc_graph* g, int32_t order);

/*
 * Sampler kernel: 0 = automatic (the default: the edge-record kernel when the
 * tree state lives in global memory, else the CSR-walk kernel with the state
 * in shared memory), 1 = CSR-walk kernel, 2 = edge-record kernel (FC_EINVAL if
 * g has no edge records: graphs without edges).  Edge records are 16 bytes
 * per CSR entry (64 bytes for weighted graphs, which also carry slot
 * thresholds) per alpha.  Both kernels draw the same random stacks, so the
 * trees are identical; only speed differs.
 * fc_sampler_last_kernel returns the kernel of the last launch on g: 1 =
 * CSR-walk, 2 = edge-record with tree membership as state flags, 3 =
 * edge-record with the in-tree bitmap in shared memory, 4 = edge-record with
 * the in-tree bitmap in global memory; 0 before any launch.
 */
fc_status fc_set_sampler_kernel(fc_graph* g, int32_t kernel);
int32_t fc_sampler_last_kernel(const fc_graph* g);

/*
 * How the edge-record kernel erases a cycle that closes on a walker's own
 * path (Wilson's loop erasure = popping the stacks of the cycle's vertices):
 * 1 = always walk the cycle through the next pointers (one dependent load per
 * vertex), 2 = when the cycle lies within the walker's last 8 path vertices,
 * pop it from shared memory at once (longer cycles are walked), 0 = automatic
 * (the default: 2 when the mean degree is below 8, where walks loop often,
 * else 1).  Affects speed only, never results.
 */
fc_status fc_set_sampler_pops(fc_graph* g, int32_t mode);

/*
 * Where the edge-record kernel keeps tree membership: 1 = a flag bit in each
 * vertex's state word (the claiming CAS reads it), 2 = a per-tree in-tree
 * bitmap in shared memory (FC_EINVAL at sampling when n/8 bytes do not fit
 * next to the walker arrays), 3 = a per-tree bitmap in global memory, 0 =
 * automatic (the default: shared memory when it fits and fc_set_sampler_shape
 * does not force global tree state, else flags).  With a bitmap, claims on
 * vertices already in the tree touch no state word and no edge record.
 * Affects speed only, never results.
 */
fc_status fc_set_sampler_bitmap(fc_graph* g, int32_t mode);

/*
 * CTAs per tree of the edge-record kernel: 1, 2, 4 or 8 CTAs of a
 * thread-block cluster share one tree (its walkers, start vertices and, with
 * the shared-memory bitmap, the bitmap split over their shared memories); 0 =
 * automatic (the default: the smallest power of two up to 8 that lets a
 * launch of few trees occupy the GPU; with fc_set_sampler_bitmap(2), grown
 * until the bitmap's share fits).  A global-memory bitmap runs with 1.
 * fc_sampler_last_cluster returns the value used by the last launch.
 * Affects speed only, never results.
 */
fc_status fc_set_sampler_cluster(fc_graph* g, int32_t ctas_per_tree);
int32_t fc_sampler_last_cluster(const fc_graph* g);

/*
 * Diagnostic per-iteration counters of the last fc_sample_usts on g, summed
 * over walkers and trees: [0] walker iterations, [1] claims at stack entry 0,
 * [2] tree hits, [3] tree-hit confirmations, [4] conflict waits, [5] waits
 * after a release, [6] releases, [7] pop steps, [8] tops computed at entry
 * k > 0, [9] idle-lane iterations.  For the edge-record kernel [1] counts
 * every successful claim (any k) and [3] counts re-reads of a vertex whose
 * owner has already moved on (its path joined the tree or was released).
 * out: host uint64[count], count >= 10.
 * The counters are compiled in only when the library is built with
 * FC_WILSON_COUNTERS=1 (they cost registers); otherwise they read 0.
 * Synchronous.
 */
fc_status fc_sampler_counters(fc_graph* g, uint64_t* out, int32_t count);

/* Launch shape used by the last fc_sample_usts on g (host pointers, may be NULL). */
fc_status fc_sampler_last_shape(const fc_graph* g, int32_t* walkers_per_tree, int32_t* regs, int32_t* ctas);

/*
 * Sample tau spanning trees of G* rooted at u* for EVERY alpha of the graph
 * (Algorithm 1's sampling loop; Algorithm 2 per tree) and aggregate them.
 * Tree t of alpha index a uses the random stacks
 *   Philox4x32-10(counter = (k, v, tree_offset + t, a), key = (seed_lo, seed_hi)),
 * so the trees, and therefore every output, are a pure function of
 * (graph, alphas, seed, tree index) -- independent of launch shape and of how
 * trees are split across calls or GPUs.
 * Outputs (device; NULL skips an optional one):
 *   R        uint32[n_alpha * n]   R[a*n + v] += #trees containing edge {u*, v}
 *            (Prop. 1; accumulated, NOT cleared: zero it before the first call)
 *   C        uint32[n_alpha * n]   C[a*n + v] += #trees whose first stack entry
 *            of v selects u* (control-variate covariate; accumulated) -- optional
 *   parents  int32[n_alpha * tau * n] parent of v in tree t of alpha a at
 *            [(a*tau + t)*n + v], u* = n -- optional (test / analysis mode)
 *   steps_out uint64[n_alpha * tau] stack entries consumed by each tree
 *            (= departures of the sequential algorithm) -- optional
 * max_steps_per_tree: watchdog on the iterations of each walker (0 = default
 * 8 n + 2^20; graphs from fc_build_rooted: 2^26 + 64 n, since walks on G have
 * a single exit); exceeding it aborts the launch with FC_ETIMEOUT.
 * Requires tau >= 0, tree_offset >= 0, tree_offset + tau <= 2^32.
 * Synchronises `stream` (reads the device error word).
 */
fc_status fc_sample_usts(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                         uint32_t* C, int32_t* parents, uint64_t max_steps_per_tree,
                         uint64_t* steps_out, void* stream);

/*
 * fc_sample_usts with one more optional output (NULL skips it):
 *   visits   uint64[n_alpha * n]   visits[a*n + v] += departures from v in each
 *            tree (its popped stack entries plus the one that gives its tree
 *            edge; accumulated).  The count does not depend on the start order
 *            (cycle popping).  Its mean per tree is deg*(v) Omega[v, v] on G*
 *            and d_w(v) r(root, v) on a graph from fc_build_rooted, where the
 *            root departs once per tree (the visits of a walk from v killed at
 *            the root: its Green's function).  Sum over v = steps_out per tree.
 * Everything else as fc_sample_usts.  Synchronises `stream`.
 */
fc_status fc_sample_usts_ex(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R, uint32_t* C,
                            int32_t* parents, uint64_t* visits, uint64_t max_steps_per_tree, uint64_t* steps_out,
                            void* stream);

/*
 * fc_sample_usts_ex with the forest of every tree (NULL skips an output):
 *   roots    int32 [rows][n]   roots[t][v] = the root of v's tree in the rooted
 *            spanning forest of G that tree t of G* leaves without u* (the
 *            vertex on v's path to u* whose parent is u*); by the matrix-forest
 *            theorem (Sec. 2) P(roots[t][v] = u) = Omega[u, v]
 *   depths   int32 [rows][n]   the number of edges from v to its root
 * rows and indexing as parents (n_alpha * tau rows, or tau rows of the union
 * for a batch).  The edge-record kernel without clusters writes both as
 * vertices join the tree, with no pass over the parents; otherwise they come
 * from fc_tree_roots on the parents (allocated internally when parents is
 * NULL).  Everything else as fc_sample_usts_ex.  Synchronises `stream`.
 */
fc_status fc_sample_usts_forest(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                                uint32_t* C, int32_t* parents, int32_t* roots, int32_t* depths, uint64_t* visits,
                                uint64_t max_steps_per_tree, uint64_t* steps_out, void* stream);

/*
 * fc_sample_usts without the synchronising error read-back, for enqueueing on
 * a stream that is being captured into a CUDA graph (the persistent sampling
 * launch, its memsets and the combinations after it become graph nodes).
 * Device-side errors stay in the graph's error word until fc_sampler_check.
 * The sampler's scratch buffer must already be large enough: make one
 * uncaptured fc_sample_usts call with the same graph and tau first (else
 * FC_EINVAL during capture).
 */
fc_status fc_sample_usts_async(fc_graph* g, uint64_t seed, int64_t tau, int64_t tree_offset, uint32_t* R,
                               uint32_t* C, int32_t* parents, uint64_t max_steps_per_tree, uint64_t* steps_out,
                               void* stream);

/* Read and clear the device error word of g (synchronises `stream`); the
 * status an fc_sample_usts call would have returned. */
fc_status fc_sampler_check(fc_graph* g, void* stream);

/*
 * Rao-Blackwellised estimate of diag(Omega) from sampled trees (an estimator
 * on the samples of Prop. 1, not in the paper).  With the parents of every
 * other vertex fixed, v's parent is u* with probability
 *   1 / (1 + alpha * sum of w_vw over neighbours w outside v's subtree),
 * which is unbiased for Omega[v, v] and has at most the variance of the
 * indicator "parent(v) = u*".  fc_rb_accumulate adds, for each of the T trees
 * in parents (device int32 [T][n], parent n = u*, as written by
 * fc_sample_usts), floor(value * 2^48 + 1/2) to acc[v] (device uint64 [n],
 * caller-owned, accumulates; totals do not depend on the order of the trees).
 * alpha_idx selects the alpha of g (batches: each vertex's graph alpha).
 * Values are computed in FP64 with one rounding per operation, the sum over
 * v's CSR row in order.  FC_EINVAL if a parent is out of range or the parents
 * do not form spanning trees of G* rooted at u*.  Synchronous.  fc_rb_diag
 * writes diag_out[v] = acc[v] / (2^48 T) (device double [n]), asynchronously.
 */
fc_status fc_rb_accumulate(fc_graph* g, int32_t alpha_idx, const int32_t* parents, int64_t T, uint64_t* acc,
                           void* stream);
fc_status fc_rb_diag(const uint64_t* acc, int32_t n, int64_t T, double* diag_out, void* stream);

/*
 * Forest farness (Eq. 3) and closeness (Def. 2) of the vertices of g from a
 * given estimate diag (device double [n]; batches: per graph).  Either output
 * may be NULL.  Asynchronous.
 */
fc_status fc_farness_from_diag(fc_graph* g, const double* diag, double* farness_out, double* closeness_out,
                               void* stream);

/*
 * Group forest closeness (Sec. 5, Algorithm 3): the greedy group S of k
 * vertices for group forest farness rho(S) = tr((L*_{-S})^{-1}) (L* the
 * Laplacian of G*, rows and columns of S removed, u* kept).  The first vertex
 * minimises Omega_vv (highest individual forest closeness); each further
 * vertex maximises ||M e_v||^2 / M_vv over V \ S with M = (L*_{-S})^{-1},
 * followed by the rank-one downdate of M.  Ties go to the smallest id.
 * Omega = (I + alpha_a L)^{-1} is solved with fc_solve at rel_tol (FP64
 * residual), then M is kept as a dense FP64 (n+1) x (n+1) matrix on the
 * device: about 16 (n+1)^2 bytes plus the solver's scratch; FC_ENOMEM when
 * that exceeds 90% of the free device memory.
 * Single graphs only (FC_EINVAL for batches); 1 <= k <= n.
 * S_out: device int32 [k], the chosen vertices in order.  farness_out:
 * device double [k] (may be NULL), farness_out[i] = rho(S[0..i]).
 * Synchronises `stream`.
 */
fc_status fc_group_closeness(fc_graph* g, int32_t alpha_idx, int32_t k, double rel_tol, int32_t* S_out,
                             double* farness_out, void* stream);

/*
 * Solve (I + alpha_a L) x_j = b_j for n_rhs right-hand sides by Jacobi-
 * preconditioned CG with FP32 inner iterations and FP64 residual / iterative
 * refinement (the paper's ground truth uses CG at tolerance 1e-9, Sec. 6.1;
 * Algorithm 1's pivot solve is a system in the same matrix, see
 * fc_pivot_solve).  b, x: FP64 [n_rhs * n], column j at offset j*n.  x is
 * used as the initial guess (zero it for x0 = 0).  Stops when every
 * ||b_j - A x_j||_2 <= rel_tol ||b_j||_2 (FP64 residual) or after max_iter
 * total inner iterations (FC_ENOCONV; best x kept).  iters_out (host, may be
 * NULL) receives the inner iterations used.  Synchronises `stream`.
 */
fc_status fc_solve(fc_graph* g, int32_t alpha_idx, const double* b, double* x, int32_t n_rhs,
                   double rel_tol, int32_t max_iter, int32_t* iters_out, void* stream);

/*
 * Algorithm 1's pivot solve: x = L*^+ (e_{u*} - 1/(n+1) 1), the mean-zero
 * solution of L* x = e_{u*} - 1/(n+1) 1 on G*.  Computed as the grounded
 * system (I + alpha L) y = -1/(n+1) 1 (x(u*) := 0, via fc_solve) followed by
 * the shift to zero mean.  x: FP64 device [n+1], x[n] = x(u*).
 * Synchronises `stream`.
 */
fc_status fc_pivot_solve(fc_graph* g, int32_t alpha_idx, double* x, double rel_tol, int32_t max_iter,
                         int32_t* iters_out, void* stream);

/*
 * Combination, farness and closeness for alpha index a (Algorithm 1's fill
 * step, Eq. 3, Def. 2), FP64 throughout:
 *   plain:      d_v = R[v]/tau                                  (Prop. 1)
 *   with pivot: d_v = R[v]/tau - x(u*) + 2 x(v) + (n+2)/(n+1)^2
 *               (the fill step yields diag(L*^+) on V; (L*^+)[V,V] =
 *                Omega - (n+2)/(n+1)^2 J adds the constant back)
 *   with C and g_pred (control variate, not in the paper):
 *               d_v -= beta_v (C[v]/tau - p_v),
 *               beta_v = (1 - clip(g_v, p_v, 1)) / (1 - p_v)
 *               (a g_v that is NaN counts as p_v: every g_pred keeps the
 *                estimator unbiased)
 *   farness_v = n d_v + sum_w d_w - 2;   closeness_v = n / farness_v.
 * R, C: the alpha-a slices (n entries each).  C, g_pred (float[n]) and x_pivot
 * (double[n+1]) may be NULL; C and g_pred must be both set or both NULL.
 * diag_out/farness_out/closeness_out: FP64 device [n] (farness/closeness may be
 * NULL).  tau >= 1.  Asynchronous (no sync).
 */
fc_status fc_forest_farness(fc_graph* g, int32_t alpha_idx, const uint32_t* R, const uint32_t* C,
                            const float* g_pred, const double* x_pivot, int64_t tau, double* diag_out,
                            double* farness_out, double* closeness_out, void* stream);

/*
 * fc_forest_farness for callers that must not allocate device memory -- for
 * example code under a memory manager that forbids allocations it does not
 * make itself, or a serving loop whose device memory is fixed once at
 * start-up.  Same arguments,
 * layouts and results as fc_forest_farness; the only difference is where the
 * temporary per-block sums live: fc_forest_farness takes them from the
 * stream-ordered pool, this entry point uses a fixed device array compiled
 * into the library (128 KiB, held on every GPU that loads the library until
 * the process exits).  It calls no cudaMalloc/cudaFree or other allocating
 * routine.  The paper has no counterpart: this is an engineering variant.
 *   - n must be <= 4194304 (2^22); larger graphs get FC_EINVAL.
 *   - The graph's device must be the current device; batches of graphs
 *     (fc_build_batch) are rejected with FC_EINVAL.
 *   - Each call looks up the array's address on the current device
 *     (cudaGetSymbolAddress, a host-side lookup; nothing is cached) and only
 *     launches kernels, so the call can be captured into a CUDA graph.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (different streams, or several host threads) race and give wrong
 *     results.  Serialise them (one stream, or events).
 *   - The array needs no clearing: each call writes every entry it reads.
 * Asynchronous (no sync).
 */
fc_status fc_forest_farness_noalloc(fc_graph* g, int32_t alpha_idx, const uint32_t* R, const uint32_t* C,
                                    const float* g_pred, const double* x_pivot, int64_t tau,
                                    double* diag_out, double* farness_out, double* closeness_out,
                                    void* stream);

/*
 * Visit estimate of diag(Omega) (not in the paper; an estimator on the same
 * samples as Prop. 1): diag_out[v] = visits[a*n + v] / (tau deg*(v)), with
 * visits from fc_sample_usts_ex (departures from v summed over tau trees of
 * alpha index a) and deg*(v) = fl(1 + fl(alpha d_w(v))).  In Wilson's
 * algorithm the departures from v do not depend on the start order, and with
 * v as the first start vertex they are the visits to v of a walk from v
 * killed at u*, whose mean is the Green's function deg*(v) r_{G*}(u*, v) =
 * deg*(v) Omega[v, v]: unbiased, and on BA and R-MAT graphs its per-tree
 * variance is tens of times below the indicator's.  Farness and closeness
 * follow with fc_farness_from_diag.  visits: device uint64 [n_alpha * n];
 * diag_out: device double [n]; batches use each vertex's graph alpha.
 * FC_EINVAL for graphs from fc_build_rooted.  Asynchronous.
 */
fc_status fc_visit_diag(fc_graph* g, int32_t alpha_idx, const uint64_t* visits, int64_t tau, double* diag_out,
                        void* stream);

/*
 * Exact probability p_v that one stack entry of v selects u* (the selector's
 * discrete probability, 1/deg*(v) up to 2^-52), FP64 device [n].  Asynchronous.
 */
fc_status fc_p_root(fc_graph* g, int32_t alpha_idx, double* p_out, void* stream);

/*
 * Learned control variate (not in the paper).  A network g(x) = p + (1 - p)
 * sigmoid(w2 . relu(W1 x + b1) + b2) predicts Omega_vv from the features
 *   x = (log(1 + deg v), log(1 + alpha d_w(v)), log(1 + sum_{u in N(v)} deg u), log alpha),
 * p = p_v (fc_p_root), 128 hidden units.  Parameters: FP32 master vector of
 * fc_mlp_param_count() = 769 floats, W1[128][4] | b1[128] | w2[128] | b2; the
 * kernels use them rounded to BF16 and accumulate in FP32.  Its output feeds
 * g_pred of fc_forest_farness; any output keeps the estimator unbiased.
 */
int32_t fc_mlp_param_count(void);

/* Features of every vertex for alpha index a: X float32 device [n][4].  Async. */
fc_status fc_vertex_features(fc_graph* g, int32_t alpha_idx, float* X, void* stream);

/* Prediction g_out float32 device [n] from features X [n][4].  Async. */
fc_status fc_mlp_forward(fc_graph* g, int32_t alpha_idx, const float* X, const float* params, float* g_out,
                         void* stream);

/*
 * Mean squared error loss(y) = mean_v (g_v - y_v)^2 and its gradient with
 * respect to the (BF16-rounded) parameters.  y float32 device [n]; grad float32
 * device [769]; loss float32 device [1] (may be NULL).  Deterministic
 * (fixed-order reductions).  Allocates temporary device memory.  Async.
 */
fc_status fc_mlp_loss_grad(fc_graph* g, int32_t alpha_idx, const float* X, const float* y, const float* params,
                           float* grad, float* loss, void* stream);

/*
 * fc_mlp_loss_grad scaled and accumulated, for training on several graphs:
 *   grad = (accumulate ? grad : 0) + weight * dloss/dparams,
 *   loss = (accumulate ? loss : 0) + weight * loss   (loss may be NULL).
 * Calling it once per graph with weight 1/#graphs (accumulate = 0 for the
 * first) leaves the mean gradient over the graphs in grad, ready for
 * fc_mlp_adam.  FC_EINVAL for a weight that is not finite.  Deterministic;
 * allocates temporary device memory.  Async.
 */
fc_status fc_mlp_loss_grad_acc(fc_graph* g, int32_t alpha_idx, const float* X, const float* y,
                               const float* params, float weight, int32_t accumulate, float* grad, float* loss,
                               void* stream);

/*
 * One Adam step (Kingma & Ba, bias-corrected; step is 1-based) on count
 * parameters, all device pointers.  Async.
 */
fc_status fc_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t count, int32_t step, float lr,
                      float beta1, float beta2, float eps, void* stream);

/*
 * Tree-path aggregation.  For T sampled trees given as parent arrays
 * (int32 device [T][n], u* = n, as written by fc_sample_usts), computes for
 * every vertex its forest root -- the vertex on its path whose parent is u* --
 * and its depth below that root (0 for roots), by pointer jumping over all
 * trees at once (O(log depth) rounds).  roots, depth: int32 device [T][n]
 * (depth may be NULL).  FC_EINVAL if some parent array is not a spanning tree rooted at u*.
 * By the matrix-forest theorem (Sec. 2), P(root(v) = u) = Omega[u, v].
 * Allocates temporary device memory.  Synchronises `stream`.
 */
fc_status fc_tree_roots(const int32_t* parents, int32_t n, int64_t T, int32_t* roots, int32_t* depth,
                        void* stream);

/*
 * Root-frequency counts for k query vertices: counts[q][v] += #{t : roots[t][v]
 * == queries[q]} (uint32 device [k][n], accumulated).  counts/T estimates the
 * column Omega[queries[q], :] without bias; the diagonal entry equals the
 * u*-edge count R.  Allocates temporary device memory.  Synchronises `stream`.
 */
fc_status fc_root_counts(const int32_t* roots, int32_t n, int64_t T, const int32_t* queries, int32_t k,
                         uint32_t* counts, void* stream);

/*
 * ---- Electrical closeness on G (Sec. 3) --------------------------------------
 * The paper's forest algorithm transfers an algorithm for diag(L^+) of a
 * connected graph G to G*; that algorithm rests on three facts (Sec. 3):
 * (i) the electrical closeness of u needs only L^+[u, u] and tr(L^+); (ii)
 * one Laplacian solve gives the column x = L^+ e_u of a pivot u, and with the
 * effective resistances r(u, v) Eq. 2 gives every diagonal entry,
 *   L^+[v, v] = r(u, v) - x[u] + 2 x[v];
 * (iii) r(u, v) is estimated from uniform spanning trees of G (Kirchhoff).
 * Electrical farness and closeness follow Def. 2 with r in place of the
 * forest distance: farness(v) = sum_w r(v, w) = n L^+[v, v] + tr(L^+),
 * closeness(v) = n / farness(v).  The calls below are that pipeline:
 *   fc_build_rooted -> fc_sample_usts -> fc_resistance_accumulate
 *   -> fc_laplacian_solve -> fc_electrical_closeness.
 */

/*
 * Build G (not G*) for uniform spanning trees rooted at the pivot `root`:
 * Wilson's walks on G leave v to neighbour j with probability w_vj / d_w(v)
 * and have the root as their only exit.  The graph is represented like G*
 * with u* joined to the root alone, so fc_sample_usts on it samples trees
 * whose parent arrays hold the root's parent as n and a uniform spanning tree
 * of G (probability proportional to the product of its edge weights) on the
 * other vertices; R counts the root in every tree, C is meaningless.
 * Random stacks (fc_sample_usts, alpha index 0): entry k of v != root with
 * Philox words o0..o3, u53 and U as in fc_build_augmented:
 *   unweighted: neighbour floor(o2 d / 2^32);
 *   weighted:   x = fl(U S_d), clamped below S_d; the first j with x < S_j
 *               (S_j the FP64 left-to-right prefix of the row's weights);
 * the root's every entry goes to n.  steps_out counts the root's one step.
 * Also builds the root's breadth-first tree (the fixed paths of the resistance
 * estimator): the parent of v is its smallest-id neighbour one level closer
 * to the root.  The sampler's automatic choices differ from G*'s because
 * walks on G are long and cross each other: start vertices in the reverse of
 * that tree's breadth-first order (fc_set_start_order: 1 selects it, 0 the
 * breadth-first order itself), at most 128 walkers per tree, and tree
 * membership as state flags (several CTAs per SM); as for every launch
 * shape and order, the trees do not depend on them.
 * CSR contract as fc_build_augmented; n >= 2, 0 <= root < n;
 * FC_EINVAL if G is not connected (electrical closeness is defined on
 * connected graphs).  Synchronises `stream`.
 */
fc_status fc_build_rooted(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx, const float* w,
                          int32_t root, uint32_t flags, void* stream, fc_graph** out);

/*
 * The root's breadth-first tree of a graph from fc_build_rooted: parent_out
 * int32 device [n] (-1 at the root), depth_out int32 device [n] (either may
 * be NULL).  Asynchronous.
 */
fc_status fc_bfs_tree(const fc_graph* g, int32_t* parent_out, int32_t* depth_out, void* stream);

/*
 * Effective-resistance path sums (Sec. 3 insight (iii); Kirchhoff's current
 * theorem).  For each of the T trees in parents (device int32 [T][n], as
 * written by fc_sample_usts on a graph from fc_build_rooted: the root's entry
 * n, every other entry a neighbour), and every vertex v, with
 * (x, b(x)) the edges of v's path in the breadth-first tree from v to the root:
 *   S_T(v) = sum over that path, from v upward, of
 *            ( [tree parent of x is b(x), x ancestor-or-self of v in the tree]
 *            - [tree parent of b(x) is x, b(x) ancestor-or-self of v] ) / w(x, b(x))
 * (E[S_T(v)] = r(root, v): the tree path from v to the root crosses an edge
 * a -> b with a probability whose net value is the unit current from v to the
 * root on that edge).  S_T(v) is summed in FP64 in path order, one rounding
 * per addition, 1 / w one FP64 division of the FP32 weight; acc[v] (device
 * int64 [n], caller-owned, accumulates) += floor(S_T(v) 2^32 + 1/2), so
 * totals do not depend on the order of the trees.  Work per tree: the sum of
 * the vertices' depths in the breadth-first tree.  FC_EINVAL for a graph not
 * from fc_build_rooted or parent arrays that are not spanning trees of G
 * rooted at the root.  Allocates temporary device memory.  Synchronous.
 */
fc_status fc_resistance_accumulate(fc_graph* g, const int32_t* parents, int64_t T, int64_t* acc, void* stream);

/*
 * x_j = L^+ b_j for n_rhs right-hand sides on a graph from fc_build_rooted
 * (L the Laplacian of the connected G): b is projected onto the complement
 * of span(1), L x = b solved by fc_solve's CG (Jacobi preconditioner d_w,
 * FP32 inner / FP64 residual and refinement to rel_tol), and x shifted to
 * zero mean.  b, x: FP64 device [n_rhs * n], column j at offset j*n; x is
 * the initial guess.  FC_ENOCONV after max_iter inner iterations (best x
 * kept).  With b = e_root this is the pivot column of insight (ii).
 * Allocates temporary device memory.  Synchronises `stream`.
 */
fc_status fc_laplacian_solve(fc_graph* g, const double* b, double* x, int32_t n_rhs, double rel_tol,
                             int32_t max_iter, int32_t* iters_out, void* stream);

/*
 * Electrical closeness from T trees and the pivot column x_pivot = L^+ e_root
 * (device double [n], fc_laplacian_solve), FP64 throughout.  Exactly one of
 * two estimates of r(root, v) is given:
 *   acc     (device int64 [n], fc_resistance_accumulate): the Kirchhoff path
 *           sums, r^ = acc[v] / (2^32 T);
 *   visits  (device uint64 [n], fc_sample_usts_ex on the rooted graph): the
 *           departures from v, r^ = visits[v] / (T d_w(v)), 0 at the root (not
 *           in the paper: the Green's-function identity; no parent arrays and
 *           no aggregation pass, and on BA and road-like graphs several times
 *           smaller per-tree variance than the path sums).
 * Then
 *   r^(root, v)                                           -> resist_out
 *   L^+[v, v]   = r^ - x[root] + 2 x[v]     (Eq. 2)       -> diag_out
 *   farness_v   = n L^+[v, v] + sum_w L^+[w, w]           -> farness_out
 *   closeness_v = n / farness_v             (Def. 2)      -> closeness_out
 * Outputs device double [n]; all but diag_out may be NULL.  T >= 1.
 * Allocates temporary device memory.  Asynchronous.
 */
fc_status fc_electrical_closeness(fc_graph* g, const int64_t* acc, const uint64_t* visits, int64_t T,
                                  const double* x_pivot, double* resist_out, double* diag_out, double* farness_out,
                                  double* closeness_out, void* stream);

/*
 * Top-k ranking (Sec. 6.1): the k vertices with the smallest diag values
 * (= highest forest closeness by Eq. 3), ascending, ties by ascending vertex
 * id.  diag: FP64 device [n]; idx_out: int32 device [k]; 1 <= k <= n.
 * Allocates temporary device memory.  Synchronises `stream`.
 */
fc_status fc_top_k(const double* diag, int32_t n, int32_t k, int32_t* idx_out, void* stream);

/*
 * Number of trees of Algorithm 1: ceil(log(2m/delta) / (2 (1-kappa)^2 eps^2)),
 * natural log (Hoeffding, proof of Thm. 1).  Returns -1 for arguments outside
 * 0 < eps < 1, 0 < delta < 1, 0 < kappa < 1, m >= 1.
 */
int64_t fc_tau_for(double eps, double delta, double kappa, int64_t m);

/*
 * Diagnostic: out[i] = the vertex selected by stack entry ks[i] of vertex
 * verts[i] in tree `tree` of alpha index a (same random stacks and selector as
 * fc_sample_usts; n = u*).  verts: int32 device [count] (each in [0, n)),
 * ks: uint32 device [count], out: int32 device [count].  Asynchronous.
 */
fc_status fc_stack_entries(fc_graph* g, int32_t alpha_idx, uint64_t seed, uint32_t tree, int64_t count,
                           const int32_t* verts, const uint32_t* ks, int32_t* out, void* stream);

/*
 * Work counters of the last fc_sample_usts call on g (host pointers, either may
 * be NULL): stack pops summed over the trees, and departures actually executed
 * (including walk steps repeated after a walker released its path).
 * Synchronous.
 */
fc_status fc_sampler_stats(fc_graph* g, uint64_t* pops, uint64_t* departures);

/*
 * Number of CUDA kernels this library has launched in the process so far
 * (diagnostic: count launches in a region by differencing).
 */
uint64_t fc_launch_count(void);

/*
 * fc_sample_usts keeps its per-tree state in one process-wide device buffer
 * per GPU, grown on demand and reused by every graph.  This frees those
 * buffers (synchronises the device).  Graphs stay valid.
 */
fc_status fc_release_scratch(void);

/* Release the graph and all device memory it owns (NULL is a no-op). */
void fc_destroy(fc_graph* g);

/* Static description of a status code. */
const char* fc_status_str(fc_status s);

/* Detail of the last failure on the calling host thread ("" if none). */
const char* fc_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* FC_H_ */
