/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, slow, sequential restatement of the sampling part of the method:
 * Wilson's algorithm on the augmented graph G* rooted at the universal vertex
 * u* (Algorithm 2, App. B; used by Algorithm 1, Sec. 4.2), with the random
 * choices drawn from counter-based "random stacks".  It shares no code with the
 * CUDA path; only tests/, the smoke check and the bench's CPU-baseline leg load
 * it.  Compile with -ffp-contract=off so that every floating-point operation is
 * the single IEEE-754 operation written here.
 *
 * Augmented graph G* (Sec. 4.1): V' = V + {u*}, u* has index n; every edge of G
 * keeps its endpoints and has weight alpha * w_e; every vertex v has an extra
 * edge {v, u*} of weight 1.  The walk at v therefore leaves to u* with
 * probability 1 / deg*(v) and to neighbour j with alpha * w_vj / deg*(v), where
 * deg*(v) = 1 + alpha * d_w(v).
 *
 * Random stack of vertex v in tree t (stack entry k = the k-th departure from v
 * in that tree): Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *   counter = (k, v, t_global, alpha_idx), key = (seed_lo, seed_hi).
 * Slot selection from the output words (o0, o1, o2, o3); slot 0 = u*, slot
 * j >= 1 = the j-th neighbour in CSR order.  U = ((o0 << 21) | (o1 >> 11)) * 2^-53
 * (53 random bits, exact in FP64).
 *   unweighted: t = fl(1 + fl(alpha * d)); x = fl(U * t), if x >= t then x = the
 *               largest double < t; x < 1 selects u*, otherwise
 *               slot = 1 + floor(o2 * d / 2^32) (uniform neighbour).
 *   weighted:   thresholds t_0 = 1, t_j = fl(1 + fl(alpha * S_j)),
 *               S_j = fl(S_{j-1} + w_j), S_0 = 0; x = fl(U * t_d), clamped below
 *               t_d as above; slot = the first j with x < t_j.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---- Philox4x32-10 as published (SC'11, Sec. 4 / Table 2) ---------------- */
static void philox_round(uint32_t x[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x[1] ^ k[0];
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x[3] ^ k[1];
    uint32_t y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(x, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

/* Batch helper for tests: out[4*i + j] = word j of Philox(ctr_i, key). */
void orc_philox_batch(int64_t count, const uint32_t* ctrs, uint64_t seed, uint32_t* out) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < count; ++i) orc_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

/* ---- one stack entry ---------------------------------------------------- */
typedef struct {
    int32_t n;
    const int64_t* rowptr;
    const int32_t* colidx;
    const double* S;      /* per-nnz FP64 prefix of the row's weights, or NULL */
    double alpha;
    const double* alpha_v; /* per-vertex alpha (a batch of graphs as one union), or NULL */
    uint32_t alpha_idx;
    uint32_t key[2];
} orc_graph;

static double below(double t) {
    /* largest double strictly below a positive finite t */
    return nextafter(t, 0.0);
}

/* Returns the vertex chosen by stack entry k of v in tree tg (n means u*). */
static int32_t stack_entry(const orc_graph* g, int32_t v, uint32_t k, uint32_t tg) {
    uint32_t ctr[4] = {k, (uint32_t)v, tg, g->alpha_idx};
    uint32_t o[4];
    orc_philox4x32_10(ctr, g->key, o);
    const int64_t b = g->rowptr[v];
    const int64_t d = g->rowptr[v + 1] - b;
    const double alpha = g->alpha_v ? g->alpha_v[v] : g->alpha;
    int64_t slot;
    const uint64_t u53 = ((uint64_t)o[0] << 21) | (uint64_t)(o[1] >> 11);
    const double U = (double)u53 * 0x1.0p-53;
    if (g->S == NULL) {
        const double t = 1.0 + alpha * (double)d;
        double x = U * t;
        if (x >= t) x = below(t);
        if (x < 1.0) slot = 0;
        else slot = 1 + (int64_t)(((uint64_t)o[2] * (uint64_t)d) >> 32);
    } else {
        const double t_last = d > 0 ? 1.0 + alpha * g->S[b + d - 1] : 1.0;
        double x = U * t_last;
        if (x >= t_last) x = below(t_last);
        slot = 0;
        if (!(x < 1.0)) {
            slot = d; /* fallback; the loop below always finds a smaller j */
            for (int64_t j = 1; j <= d; ++j) {
                const double tj = 1.0 + alpha * g->S[b + j - 1];
                if (x < tj) { slot = j; break; }
            }
        }
    }
    if (slot == 0) return g->n;
    return g->colidx[b + slot - 1];
}

/* Ascending-degree order, ties by vertex id (Algorithm 2, vertex reordering). */
static void ascending_degree_order(int32_t n, const int64_t* rowptr, int32_t* order) {
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = rowptr[v + 1] - rowptr[v];
        if (d > maxd) maxd = d;
    }
    int64_t* cnt = (int64_t*)calloc((size_t)maxd + 2, sizeof(int64_t));
    for (int32_t v = 0; v < n; ++v) cnt[rowptr[v + 1] - rowptr[v] + 1]++;
    for (int64_t d = 1; d <= maxd + 1; ++d) cnt[d] += cnt[d - 1];
    for (int32_t v = 0; v < n; ++v) order[cnt[rowptr[v + 1] - rowptr[v]]++] = v;
    free(cnt);
}

/* Per-row FP64 prefix sums of the weights, summed left to right. */
void orc_row_prefix(int32_t n, const int64_t* rowptr, const float* w, double* S) {
    for (int32_t v = 0; v < n; ++v) {
        double s = 0.0;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            s = s + (double)w[e];
            S[e] = s;
        }
    }
}

/*
 * Sample trees t = 0..tau-1 (global index tree_offset + t) of G* rooted at u*.
 *   R[v]       += number of trees in which {u*, v} is a tree edge
 *   C[v]       += number of trees whose stack entry 0 of v selects u*   (may be NULL)
 *   parents    [tau][n]: tree parent of v (n = u*)                      (may be NULL)
 *   steps      [tau]: number of stack entries consumed (= departures)  (may be NULL)
 *   visits     [n]: += departures from v, summed over the trees        (may be NULL)
 *   order      start-vertex order, NULL = ascending degree
 * Returns 0 on success, -1 on allocation failure.
 */
int orc_wilson_v(int32_t n, const int64_t* rowptr, const int32_t* colidx, const float* w,
                 double alpha, const double* alpha_v, uint32_t alpha_idx, uint64_t seed,
                 int64_t tree_offset, int64_t tau, const int32_t* order_in, uint32_t* R, uint32_t* C,
                 int32_t* parents, uint64_t* steps, uint64_t* visits);

int orc_wilson(int32_t n, const int64_t* rowptr, const int32_t* colidx, const float* w,
               double alpha, uint32_t alpha_idx, uint64_t seed, int64_t tree_offset,
               int64_t tau, const int32_t* order_in, uint32_t* R, uint32_t* C,
               int32_t* parents, uint64_t* steps) {
    return orc_wilson_v(n, rowptr, colidx, w, alpha, NULL, alpha_idx, seed, tree_offset, tau,
                        order_in, R, C, parents, steps, NULL);
}

/* As orc_wilson with an optional per-vertex alpha (alpha_v != NULL overrides
 * alpha): a batch of graphs given as one block-diagonal union, each vertex
 * carrying its own graph's alpha. */
int orc_wilson_v(int32_t n, const int64_t* rowptr, const int32_t* colidx, const float* w,
                 double alpha, const double* alpha_v, uint32_t alpha_idx, uint64_t seed,
                 int64_t tree_offset, int64_t tau, const int32_t* order_in, uint32_t* R, uint32_t* C,
                 int32_t* parents, uint64_t* steps, uint64_t* visits) {
    orc_graph g;
    g.n = n; g.rowptr = rowptr; g.colidx = colidx; g.alpha = alpha; g.alpha_idx = alpha_idx;
    g.alpha_v = alpha_v;
    g.key[0] = (uint32_t)seed; g.key[1] = (uint32_t)(seed >> 32);
    g.S = NULL;
    double* S = NULL;
    if (w != NULL) {
        S = (double*)malloc(sizeof(double) * (size_t)(rowptr[n] > 0 ? rowptr[n] : 1));
        if (!S) return -1;
        orc_row_prefix(n, rowptr, w, S);
        g.S = S;
    }
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t* in_tree = (uint8_t*)malloc((size_t)n + 1);
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint32_t* cnt = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    if (!order || !in_tree || !next || !cnt) {
        free(S); free(order); free(in_tree); free(next); free(cnt);
        return -1;
    }
    if (order_in) memcpy(order, order_in, sizeof(int32_t) * (size_t)n);
    else ascending_degree_order(n, rowptr, order);

    for (int64_t t = 0; t < tau; ++t) {
        const uint32_t tg = (uint32_t)(tree_offset + t);
        memset(in_tree, 0, (size_t)n + 1);
        memset(cnt, 0, sizeof(uint32_t) * ((size_t)n + 1));
        in_tree[n] = 1; /* T = {u*} */
        next[n] = -1;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t s = order[i];
            /* random walk from s until it hits T; overwriting next[] on every
               departure erases loops in order of appearance (last exit). */
            int32_t u = s;
            while (!in_tree[u]) {
                next[u] = stack_entry(&g, u, cnt[u], tg);
                cnt[u]++;
                u = next[u];
            }
            /* T <- T + LE(P), remembering the last vertex before u* */
            int32_t last = -1;
            u = s;
            while (!in_tree[u]) {
                in_tree[u] = 1;
                last = u;
                u = next[u];
            }
            if (last >= 0 && u == n) R[last] += 1;
        }
        if (C) {
            for (int32_t v = 0; v < n; ++v)
                if (stack_entry(&g, v, 0u, tg) == n) C[v] += 1;
        }
        if (parents) {
            for (int32_t v = 0; v < n; ++v) parents[t * (int64_t)n + v] = next[v];
        }
        if (steps) {
            uint64_t s = 0;
            for (int32_t v = 0; v < n; ++v) s += cnt[v];
            steps[t] = s;
        }
        if (visits) {
            for (int32_t v = 0; v < n; ++v) visits[v] += cnt[v];
        }
    }
    free(S); free(order); free(in_tree); free(next); free(cnt);
    return 0;
}

/* Exact probability that one stack entry of v selects u*, as a count over the
 * selector's 2^53 equally likely values of u53 (count / 2^53): the count of u53
 * with x(u53) < 1, found by bisection over the monotone map
 * u53 -> fl(u53 * 2^-53 * t) (clamped below t), where t = fl(1 + fl(alpha * d))
 * unweighted and t = fl(1 + fl(alpha * S_d)) weighted. */
double orc_p_root(int64_t d, double alpha, double S_d, int weighted) {
    const double t_last = weighted ? (d > 0 ? 1.0 + alpha * S_d : 1.0) : 1.0 + alpha * (double)d;
    /* count u53 in [0, 2^53) with x(u53) < 1 where x = fl(U t_last) clamped below t_last */
    uint64_t lo = 0, hi = (uint64_t)1 << 53; /* invariant: x(lo-1) < 1 known for lo>0; x(hi) >= 1 or hi = 2^53 */
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        double x = (double)mid * 0x1.0p-53 * t_last;
        if (x >= t_last) x = below(t_last);
        if (x < 1.0) lo = mid + 1; else hi = mid;
    }
    return (double)lo * 0x1.0p-53;
}

/* Test helper: out[i] = vertex chosen by stack entry ks[i] of verts[i] in tree tg
 * (n = u*).  Builds the weight prefix itself when w != NULL. */
int orc_stack_entries(int32_t n, const int64_t* rowptr, const int32_t* colidx, const float* w,
                      double alpha, uint32_t alpha_idx, uint64_t seed, uint32_t tg,
                      int64_t count, const int32_t* verts, const uint32_t* ks, int32_t* out) {
    orc_graph g;
    g.n = n; g.rowptr = rowptr; g.colidx = colidx; g.alpha = alpha; g.alpha_idx = alpha_idx;
    g.alpha_v = NULL;
    g.key[0] = (uint32_t)seed; g.key[1] = (uint32_t)(seed >> 32);
    g.S = NULL;
    double* S = NULL;
    if (w != NULL) {
        S = (double*)malloc(sizeof(double) * (size_t)(rowptr[n] > 0 ? rowptr[n] : 1));
        if (!S) return -1;
        orc_row_prefix(n, rowptr, w, S);
        g.S = S;
    }
    for (int64_t i = 0; i < count; ++i) out[i] = stack_entry(&g, verts[i], ks[i], tg);
    free(S);
    return 0;
}

/*
 * Wilson's algorithm on G itself, rooted at the vertex `root` (the uniform
 * spanning trees of G that the electrical-closeness algorithm samples, Sec. 3
 * insight (iii); Algorithm 2 with T = {root} at the start).  G must be
 * connected.  The walk at v leaves to neighbour j with probability
 * w_vj / d_w(v); stack entry k of v in tree t is Philox4x32-10 with
 * counter = (k, v, t_global, 0), key = (seed_lo, seed_hi), and
 *   unweighted: neighbour floor(o2 * d / 2^32) of v's row;
 *   weighted:   x = fl(U * S_d), clamped below S_d (U as above, S_j the
 *               row's FP64 weight prefix); the first j with x < S_j.
 * Outputs (each may be NULL):
 *   parents [tau][n]: the next vertex on v's tree path to the root; the root's
 *           entry is n (the root, seen as the only vertex joined to an
 *           outside vertex n)
 *   steps   [tau]: stack entries consumed (departures; the root makes none)
 *   visits  [n]: += departures from v, summed over the trees (the root's 0)
 * Returns 0, -1 on allocation failure, -2 if G is not connected.
 */
static int32_t stack_entry_rooted(const orc_graph* g, int32_t v, uint32_t k, uint32_t tg) {
    uint32_t ctr[4] = {k, (uint32_t)v, tg, 0u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, g->key, o);
    const int64_t b = g->rowptr[v];
    const int64_t d = g->rowptr[v + 1] - b;
    int64_t j;
    if (g->S == NULL) {
        j = (int64_t)(((uint64_t)o[2] * (uint64_t)d) >> 32);
    } else {
        const uint64_t u53 = ((uint64_t)o[0] << 21) | (uint64_t)(o[1] >> 11);
        const double U = (double)u53 * 0x1.0p-53;
        const double t_last = g->S[b + d - 1];
        double x = U * t_last;
        if (x >= t_last) x = below(t_last);
        j = d - 1;
        for (int64_t i = 0; i < d; ++i) {
            if (x < g->S[b + i]) { j = i; break; }
        }
    }
    return g->colidx[b + j];
}

int orc_wilson_rooted(int32_t n, const int64_t* rowptr, const int32_t* colidx, const float* w, int32_t root,
                      uint64_t seed, int64_t tree_offset, int64_t tau, const int32_t* order_in,
                      int32_t* parents, uint64_t* steps, uint64_t* visits) {
    orc_graph g;
    g.n = n; g.rowptr = rowptr; g.colidx = colidx; g.alpha = 1.0; g.alpha_idx = 0;
    g.alpha_v = NULL;
    g.key[0] = (uint32_t)seed; g.key[1] = (uint32_t)(seed >> 32);
    g.S = NULL;
    double* S = NULL;
    if (w != NULL) {
        S = (double*)malloc(sizeof(double) * (size_t)(rowptr[n] > 0 ? rowptr[n] : 1));
        if (!S) return -1;
        orc_row_prefix(n, rowptr, w, S);
        g.S = S;
    }
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t* in_tree = (uint8_t*)malloc((size_t)n + 1);
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint32_t* cnt = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    if (!order || !in_tree || !next || !cnt) {
        free(S); free(order); free(in_tree); free(next); free(cnt);
        return -1;
    }
    if (order_in) memcpy(order, order_in, sizeof(int32_t) * (size_t)n);
    else ascending_degree_order(n, rowptr, order);
    int rc = 0;
    /* connectivity: breadth-first search from the root (order[] as the queue
       is overwritten below only after the check) */
    {
        int32_t* q = (int32_t*)next; /* n + 1 slots */
        int64_t head = 0, tail = 0, seen = 1;
        memset(in_tree, 0, (size_t)n + 1);
        in_tree[root] = 1;
        q[tail++] = root;
        while (head < tail) {
            const int32_t x = q[head++];
            for (int64_t e = rowptr[x]; e < rowptr[x + 1]; ++e) {
                const int32_t y = colidx[e];
                if (!in_tree[y]) { in_tree[y] = 1; q[tail++] = y; ++seen; }
            }
        }
        if (seen != n) rc = -2;
    }
    for (int64_t t = 0; t < tau && rc == 0; ++t) {
        const uint32_t tg = (uint32_t)(tree_offset + t);
        memset(in_tree, 0, (size_t)n + 1);
        memset(cnt, 0, sizeof(uint32_t) * ((size_t)n + 1));
        in_tree[root] = 1; /* T = {root} */
        next[root] = n;
        for (int32_t i = 0; i < n && rc == 0; ++i) {
            const int32_t s = order[i];
            int32_t u = s;
            while (!in_tree[u]) {
                if (rowptr[u + 1] == rowptr[u]) { rc = -2; break; }
                next[u] = stack_entry_rooted(&g, u, cnt[u], tg);
                cnt[u]++;
                u = next[u];
            }
            u = s;
            while (rc == 0 && !in_tree[u]) {
                in_tree[u] = 1;
                u = next[u];
            }
        }
        if (parents) {
            for (int32_t v = 0; v < n; ++v) parents[t * (int64_t)n + v] = next[v];
        }
        if (steps) {
            uint64_t s = 0;
            for (int32_t v = 0; v < n; ++v) s += cnt[v];
            steps[t] = s;
        }
        if (visits) {
            for (int32_t v = 0; v < n; ++v) visits[v] += cnt[v];
        }
    }
    free(S); free(order); free(in_tree); free(next); free(cnt);
    return rc;
}
