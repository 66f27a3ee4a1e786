/*
 * ocm_oracle.c -- plain, slow, single-threaded CPU oracle for the optimal
 * cycle mean (OCM) problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this file: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
 * solver (no header, helper or constant), and every integer is exact
 * (int64 / __int128), so its answers are the parity target.
 *
 * Problem (paper Sec. 2.1, definition of cycle mean and the OCM problem): for
 * a digraph G = (V, E) with integer edge weights w, the cycle mean of a cycle
 * C is w(C)/|C|.  The *_ratio entry points take a second integer label, a
 * transit time t(e) >= 1 per edge (the "time" of a transition, Sec. 2.2), and
 * compute the optimal cycle ratio w(C)/t(C) instead; with t = 1 everywhere
 * the ratio is the mean, and every routine below reduces to its mean form.  The paper states the minimal cycle mean; this oracle works
 * in the maximising sense, lambda* = max over cycles C of w(C)/|C|, and the
 * minimising sense is obtained as  min(w) = -max(-w)  with the same critical
 * cycle.  Results are reduced rationals num/den with den > 0.
 *
 * Contents
 *   oracle_howard      Howard policy iteration, Alg. 1 (Sec. 2.4), in the
 *                      deterministic multichain reading: exact per-vertex
 *                      cycle means eta(v), values V(v) scaled by eta's
 *                      denominator, strict improvement, fixed tie-breaks.
 *   oracle_karp        Karp's O(nm) recurrence (Karp 1978), with the
 *                      super-source augmentation of Sec. 2.1 so that input
 *                      need not be strongly connected.
 *   oracle_brute       enumeration of every simple cycle (tiny graphs).
 *   oracle_tarjan_scc  strongly connected components (Sec. 2.4, Tarjan).
 *   oracle_certificate checks an answer against the LP dual of Eq. (1):
 *                      per-vertex means that never increase along an edge and
 *                      potentials under which no edge has positive reduced
 *                      weight (Prop. 2.1), plus a cycle attaining the value.
 *   oracle_howard_ratio, oracle_brute_ratio, oracle_certificate_ratio
 *                      the same three for the optimal cycle ratio.
 *   oracle_howard_single  the paper's own form of the iteration (Alg. 1 as
 *                      written): one lambda, every other policy cycle broken
 *                      each iteration (strongly connected input only).
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *   - max sense (the paper defines min); min via negated weights;
 *   - initial policy = the paper's first pass from val = 0, lambda = 0: the
 *     heaviest out-edge, ties to the smallest CSR edge index;
 *   - a vertex switches only on strict improvement (Alg. 1), ties keep it;
 *   - the root of a policy cycle is its smallest vertex (Alg. 1 MinVertex,
 *     and Sec. 3.1: the same vertex whenever the same cycle is chosen);
 *   - instead of rebuilding the policy graph around one chosen cycle
 *     (Alg. 1 "break all other cycles", Alg. 2 markMinComponent/connectGpi),
 *     every policy cycle keeps its own mean (multichain policy iteration),
 *     so input need not be strongly connected; lambda* is the largest mean of
 *     the final policy, the critical cycle that of the smallest root with it;
 *   - oracle_howard_single keeps the rebuild; where several out-edges of an
 *     unconnected vertex lead into the connected part, it takes the smallest
 *     CSR edge index among those into vertices connected at earlier levels
 *     of the backward search (the paper leaves the choice open).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

enum {
    OR_OK = 0,
    OR_ERR_ARG = -1,
    OR_ERR_CSR = -2,
    OR_ERR_NO_OUT_EDGE = -3,
    OR_ERR_RANGE = -4,
    OR_ERR_NOT_CONVERGED = -5,
    OR_ERR_NOMEM = -6,
    OR_ERR_TOO_MANY = -7,
    OR_ERR_NOT_SC = -8,
};

static int64_t gcd64(int64_t a, int64_t b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static int check_csr(int32_t n, int32_t m, const int32_t *rp, const int32_t *col) {
    if (n <= 0 || m <= 0 || !rp || !col) return OR_ERR_ARG;
    if (rp[0] != 0 || rp[n] != m) return OR_ERR_CSR;
    for (int32_t v = 0; v < n; ++v) {
        if (rp[v + 1] < rp[v]) return OR_ERR_CSR;
        if (rp[v + 1] == rp[v]) return OR_ERR_NO_OUT_EDGE;
    }
    for (int32_t e = 0; e < m; ++e)
        if (col[e] < 0 || col[e] >= n) return OR_ERR_CSR;
    return OR_OK;
}

/* weight in the maximising sense */
static inline int64_t wmax(const int32_t *w, int32_t e, int mode) {
    return mode == 0 ? (int64_t)w[e] : -(int64_t)w[e];
}

/* transit time of edge e (1 when no times are given) */
static inline int64_t tval(const int32_t *tt, int32_t e) { return tt ? (int64_t)tt[e] : 1; }

/* compare fractions a/b and c/d (b, d > 0): -1, 0, 1 */
static inline int frac_cmp(int64_t a, int64_t b, int64_t c, int64_t d) {
    i128 l = (i128)a * d, r = (i128)c * b;
    return (l > r) - (l < r);
}

/* ======================================================================== */
/* Howard policy iteration (Alg. 1), multichain reading                      */
/* ======================================================================== */

typedef struct {
    int32_t n;
    const int32_t *rp, *col, *w;
    int mode;
    int32_t *pi;        /* policy: an out-edge index per vertex            */
    int32_t *succ;      /* successor in the policy graph G_pi              */
    int32_t *cyc;       /* id of the cycle the vertex reaches              */
    int32_t *state;     /* walk colouring                                  */
    int32_t *path;      /* walk stack                                      */
    int64_t *S;         /* weight of the policy path to the cycle's root   */
    const int32_t *tt;  /* transit times (NULL: 1 on every edge)          */
    int64_t *T;         /* transit time of the path to the root            */
    i128 *V;            /* q*S - p*T : value scaled by the mean's denominator */
    int32_t ncyc;
    int32_t *cyc_root;  /* per cycle: smallest vertex on it                */
    int64_t *cyc_p, *cyc_q;  /* per cycle: reduced mean p/q                */
} howard_ws;

/* Evaluate the policy pi: find every cycle of the functional graph G_pi by
 * following successors and colouring visited vertices (Sec. 2.4: each weakly
 * connected component of G_pi holds exactly one cycle), take its root = the
 * smallest vertex, its mean W/L (ratio: W/T, T = transit time of the cycle)
 * reduced to p/q, and propagate values from the root along policy
 * predecessors (Alg. 1 value propagation):
 * V(root) = 0, V(v) = q*w(v, succ v) - p*t(v, succ v) + V(succ v),
 * i.e. V = q*S - p*T with S, T the weight and time of v's path to the root
 * (T = len for the mean). */
static void howard_evaluate(howard_ws *h) {
    int32_t n = h->n;
    for (int32_t v = 0; v < n; ++v) {
        h->succ[v] = h->col[h->pi[v]];
        h->state[v] = 0;
    }
    h->ncyc = 0;
    for (int32_t v0 = 0; v0 < n; ++v0) {
        if (h->state[v0] != 0) continue;
        int32_t top = 0, u = v0;
        while (h->state[u] == 0) {
            h->state[u] = 1;
            h->path[top++] = u;
            u = h->succ[u];
        }
        int32_t stop = top;   /* path[0..stop) still needs values */
        if (h->state[u] == 1) {
            /* new cycle: path[k..top) with path[k] == u */
            int32_t k = top - 1;
            while (h->path[k] != u) --k;
            int32_t c = h->ncyc++;
            int32_t root = u;
            int64_t W = 0, Tc = 0;
            for (int32_t j = k; j < top; ++j) {
                int32_t x = h->path[j];
                if (x < root) root = x;
                W += wmax(h->w, h->pi[x], h->mode);
                Tc += tval(h->tt, h->pi[x]);
            }
            int64_t g = gcd64(W, Tc);
            h->cyc_root[c] = root;
            h->cyc_p[c] = W / g;
            h->cyc_q[c] = Tc / g;
            /* walk the cycle backwards from the root: the root is terminal */
            h->S[root] = 0;
            h->T[root] = 0;
            h->cyc[root] = c;
            h->state[root] = 2;
            /* vertices of the cycle in order starting at root */
            int32_t cl = top - k;
            int32_t start = k;
            while (h->path[start] != root) ++start;
            for (int32_t t = cl - 1; t >= 1; --t) {
                int32_t x = h->path[k + (start - k + t) % cl];
                int32_t y = h->succ[x];
                h->S[x] = wmax(h->w, h->pi[x], h->mode) + h->S[y];
                h->T[x] = tval(h->tt, h->pi[x]) + h->T[y];
                h->cyc[x] = c;
                h->state[x] = 2;
            }
            stop = k;
        }
        /* tree part: path[0..stop) leads into a vertex with known values */
        for (int32_t j = stop - 1; j >= 0; --j) {
            int32_t x = h->path[j];
            int32_t y = h->succ[x];
            h->S[x] = wmax(h->w, h->pi[x], h->mode) + h->S[y];
            h->T[x] = tval(h->tt, h->pi[x]) + h->T[y];
            h->cyc[x] = h->cyc[y];
            h->state[x] = 2;
        }
    }
    for (int32_t v = 0; v < n; ++v) {
        int32_t c = h->cyc[v];
        h->V[v] = (i128)h->cyc_q[c] * h->S[v] - (i128)h->cyc_p[c] * h->T[v];
    }
}

/* improvement key of edge e: (eta(t), q_t*w(e) - p_t*t(e) + V(t)), t = col[e] */
static inline i128 howard_key2(const howard_ws *h, int32_t e) {
    int32_t t = h->col[e];
    int32_t c = h->cyc[t];
    return (i128)h->cyc_q[c] * wmax(h->w, e, h->mode) - (i128)h->cyc_p[c] * tval(h->tt, e) +
           h->V[t];
}

/* Is edge a better than edge b for the improvement step?  Lexicographic
 * maximum of (eta(t), key2, -edge index). */
static inline int howard_better(const howard_ws *h, int32_t a, int32_t b) {
    int32_t ca = h->cyc[h->col[a]], cb = h->cyc[h->col[b]];
    int c = frac_cmp(h->cyc_p[ca], h->cyc_q[ca], h->cyc_p[cb], h->cyc_q[cb]);
    if (c != 0) return c > 0;
    i128 ka = howard_key2(h, a), kb = howard_key2(h, b);
    if (ka != kb) return ka > kb;
    return a < b;
}

/*
 * oracle_howard
 *   n, m, rp[n+1], col[m], w[m] : CSR digraph, every vertex with out-degree >= 1
 *   mode     : 0 = maximum cycle mean, 1 = minimum cycle mean
 *   max_iter : iteration cap (<= 0: 4n + 64)
 * Outputs (pointers may be NULL where marked optional):
 *   num, den           : lambda* = num/den reduced, den > 0 (in the given mode)
 *   cycle[n], clen     : critical cycle as CSR edge indices, starting with the
 *                        policy edge of its smallest vertex
 *   eta_p, eta_q [n]   : optional, per-vertex mean of the reached policy cycle
 *                        (max sense, i.e. of -w in min mode)
 *   V [n]              : optional, final values (max sense), must fit int64
 *   policy [n]         : optional, final policy edge per vertex
 *   iters              : optional, number of improvement steps taken
 *   trace [3*tcap]     : optional, per iteration (cycles, switched, eval id)
 *   init [n]           : optional initial policy (an out-edge index of each
 *                        vertex); NULL = the first pass of Alg. 1 from val = 0,
 *                        lambda = 0.  Policy iteration reaches an optimal
 *                        policy from any start (Sec. 2.4), so a caller may
 *                        resume from an earlier policy (warm start).
 * Returns 0 or a negative OR_ERR_* code.
 */
static int howard_impl(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                       const int32_t *w, const int32_t *tt, int mode, int64_t max_iter,
                       int64_t *num, int64_t *den, int32_t *cycle, int32_t *clen,
                       int64_t *eta_p, int64_t *eta_q, int64_t *V_out, int32_t *policy,
                       int64_t *iters, int64_t *trace, int64_t tcap, const int32_t *init) {
    int rc = check_csr(n, m, rp, col);
    if (rc) return rc;
    if (tt)
        for (int32_t e = 0; e < m; ++e)
            if (tt[e] < 1) return OR_ERR_ARG;
    if (init)
        for (int32_t v = 0; v < n; ++v)
            if (init[v] < rp[v] || init[v] >= rp[v + 1]) return OR_ERR_ARG;
    if (!w || (mode != 0 && mode != 1)) return OR_ERR_ARG;
    for (int32_t e = 0; e < m; ++e)
        if (w[e] == INT32_MIN) return OR_ERR_RANGE;
    if (max_iter <= 0) max_iter = 4 * (int64_t)n + 64;

    howard_ws h;
    memset(&h, 0, sizeof h);
    h.n = n; h.rp = rp; h.col = col; h.w = w; h.mode = mode; h.tt = tt;
    size_t N = (size_t)n;
    h.pi = malloc(N * sizeof(int32_t));
    h.succ = malloc(N * sizeof(int32_t));
    h.cyc = malloc(N * sizeof(int32_t));
    h.state = malloc(N * sizeof(int32_t));
    h.path = malloc(N * sizeof(int32_t));
    h.S = malloc(N * sizeof(int64_t));
    h.T = malloc(N * sizeof(int64_t));
    h.V = malloc(N * sizeof(i128));
    h.cyc_root = malloc(N * sizeof(int32_t));
    h.cyc_p = malloc(N * sizeof(int64_t));
    h.cyc_q = malloc(N * sizeof(int64_t));
    int32_t *newpi = malloc(N * sizeof(int32_t));
    rc = OR_OK;
    if (!h.pi || !h.succ || !h.cyc || !h.state || !h.path || !h.S || !h.T || !h.V ||
        !h.cyc_root || !h.cyc_p || !h.cyc_q || !newpi) {
        rc = OR_ERR_NOMEM;
        goto done;
    }

    /* first pass from val = 0, lambda = 0: heaviest out-edge, smallest index
     * (or the caller's initial policy) */
    for (int32_t v = 0; v < n; ++v) {
        int32_t best = rp[v];
        for (int32_t e = rp[v] + 1; e < rp[v + 1]; ++e)
            if (wmax(w, e, mode) > wmax(w, best, mode)) best = e;
        h.pi[v] = init ? init[v] : best;
    }

    int64_t it = 0;
    for (;;) {
        howard_evaluate(&h);
        /* improvement (Jacobi: all vertices read the same evaluation) */
        int64_t switched = 0;
        for (int32_t v = 0; v < n; ++v) {
            int32_t best = rp[v];
            for (int32_t e = rp[v] + 1; e < rp[v + 1]; ++e)
                if (howard_better(&h, e, best)) best = e;
            int32_t cur = h.pi[v];
            int32_t cb = h.cyc[col[best]], cv = h.cyc[v];
            int c = frac_cmp(h.cyc_p[cb], h.cyc_q[cb], h.cyc_p[cv], h.cyc_q[cv]);
            int sw = c > 0 || (c == 0 && howard_key2(&h, best) > howard_key2(&h, cur));
            newpi[v] = sw ? best : cur;
            switched += sw;
        }
        if (trace && it < tcap) {
            trace[3 * it + 0] = h.ncyc;
            trace[3 * it + 1] = switched;
            trace[3 * it + 2] = it;
        }
        if (switched == 0) break;
        if (++it >= max_iter) {
            rc = OR_ERR_NOT_CONVERGED;
            goto done;
        }
        memcpy(h.pi, newpi, N * sizeof(int32_t));
    }

    /* lambda* = largest cycle mean of the final policy; critical cycle = the
     * one with the smallest root among those attaining it */
    int32_t bc = 0;
    for (int32_t c = 1; c < h.ncyc; ++c) {
        int k = frac_cmp(h.cyc_p[c], h.cyc_q[c], h.cyc_p[bc], h.cyc_q[bc]);
        if (k > 0 || (k == 0 && h.cyc_root[c] < h.cyc_root[bc])) bc = c;
    }
    if (num) *num = mode == 0 ? h.cyc_p[bc] : -h.cyc_p[bc];
    if (den) *den = h.cyc_q[bc];
    {
        int32_t r = h.cyc_root[bc], x = r, L = 0;
        do {
            if (cycle) cycle[L] = h.pi[x];
            ++L;
            x = h.succ[x];
        } while (x != r);
        if (clen) *clen = L;
    }
    for (int32_t v = 0; v < n; ++v) {
        int32_t c = h.cyc[v];
        if (eta_p) eta_p[v] = h.cyc_p[c];
        if (eta_q) eta_q[v] = h.cyc_q[c];
        if (V_out) {
            if (h.V[v] > (i128)INT64_MAX || h.V[v] < (i128)INT64_MIN) {
                rc = OR_ERR_RANGE;
                goto done;
            }
            V_out[v] = (int64_t)h.V[v];
        }
        if (policy) policy[v] = h.pi[v];
    }
    if (iters) *iters = it;

done:
    free(h.pi); free(h.succ); free(h.cyc); free(h.state); free(h.path);
    free(h.S); free(h.T); free(h.V); free(h.cyc_root); free(h.cyc_p);
    free(h.cyc_q);
    free(newpi);
    return rc;
}

int oracle_howard(int32_t n, int32_t m, const int32_t *rp, const int32_t *col, const int32_t *w,
                  int mode, int64_t max_iter, int64_t *num, int64_t *den, int32_t *cycle,
                  int32_t *clen, int64_t *eta_p, int64_t *eta_q, int64_t *V_out,
                  int32_t *policy, int64_t *iters, int64_t *trace, int64_t tcap,
                  const int32_t *init) {
    return howard_impl(n, m, rp, col, w, NULL, mode, max_iter, num, den, cycle, clen, eta_p,
                       eta_q, V_out, policy, iters, trace, tcap, init);
}

/*
 * oracle_howard_single -- Alg. 1 as the paper writes it: after every
 * improvement step, take the policy cycle of best mean (ties: smallest root,
 * "the same vertex whenever the same cycle is chosen"), keep the component of
 * the policy graph that reaches it, and connect every other vertex to it
 * ("break all other cycles ... so that all vertices have path to C", done in
 * the paper by backward reachabilities): level by level, a vertex outside the
 * connected set takes its smallest-index out-edge into the vertices
 * connected at earlier levels.  Values are then propagated from the cycle's
 * smallest vertex with the one lambda, and the improvement step switches a
 * vertex on strict improvement of q*w(e) - p*t(e) + V(t).  Every vertex must
 * reach the chosen cycle (true for strongly connected input; OR_ERR_NOT_SC
 * otherwise).  tt = transit times for the cycle ratio, NULL for the mean;
 * init = an optional start policy as in oracle_howard.
 * Outputs as oracle_howard (V and policy optional, the final policy has the
 * one cycle); iters counts improvement steps that switched a vertex.
 */
int oracle_howard_single(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                         const int32_t *w, const int32_t *tt, int mode, int64_t max_iter,
                         int64_t *num, int64_t *den, int32_t *cycle, int32_t *clen,
                         int64_t *V_out, int32_t *policy, int64_t *iters, const int32_t *init) {
    int rc = check_csr(n, m, rp, col);
    if (rc) return rc;
    if (tt)
        for (int32_t e = 0; e < m; ++e)
            if (tt[e] < 1) return OR_ERR_ARG;
    if (init)
        for (int32_t v = 0; v < n; ++v)
            if (init[v] < rp[v] || init[v] >= rp[v + 1]) return OR_ERR_ARG;
    if (!w || (mode != 0 && mode != 1)) return OR_ERR_ARG;
    for (int32_t e = 0; e < m; ++e)
        if (w[e] == INT32_MIN) return OR_ERR_RANGE;
    if (max_iter <= 0) max_iter = 4 * (int64_t)n + 64;
    howard_ws h;
    memset(&h, 0, sizeof h);
    h.n = n; h.rp = rp; h.col = col; h.w = w; h.mode = mode; h.tt = tt;
    size_t N = (size_t)n;
    h.pi = malloc(N * sizeof(int32_t));
    h.succ = malloc(N * sizeof(int32_t));
    h.cyc = malloc(N * sizeof(int32_t));
    h.state = malloc(N * sizeof(int32_t));
    h.path = malloc(N * sizeof(int32_t));
    h.S = malloc(N * sizeof(int64_t));
    h.T = malloc(N * sizeof(int64_t));
    h.V = malloc(N * sizeof(i128));
    h.cyc_root = malloc(N * sizeof(int32_t));
    h.cyc_p = malloc(N * sizeof(int64_t));
    h.cyc_q = malloc(N * sizeof(int64_t));
    int32_t *newpi = malloc(N * sizeof(int32_t));
    int32_t *level = malloc(N * sizeof(int32_t));
    int32_t *pick = malloc(N * sizeof(int32_t));
    rc = OR_OK;
    if (!h.pi || !h.succ || !h.cyc || !h.state || !h.path || !h.S || !h.T || !h.V ||
        !h.cyc_root || !h.cyc_p || !h.cyc_q || !newpi || !level || !pick) {
        rc = OR_ERR_NOMEM;
        goto done;
    }
    for (int32_t v = 0; v < n; ++v) {     /* first pass from val = 0, lambda = 0 */
        int32_t best = rp[v];
        for (int32_t e = rp[v] + 1; e < rp[v + 1]; ++e)
            if (wmax(w, e, mode) > wmax(w, best, mode)) best = e;
        h.pi[v] = init ? init[v] : best;   /* or the caller's start (warm start) */
    }
    int64_t it = 0;
    int32_t bc = 0;
    for (;;) {
        howard_evaluate(&h);
        /* the chosen cycle: best mean, smallest root */
        bc = 0;
        for (int32_t c = 1; c < h.ncyc; ++c) {
            int k = frac_cmp(h.cyc_p[c], h.cyc_q[c], h.cyc_p[bc], h.cyc_q[bc]);
            if (k > 0 || (k == 0 && h.cyc_root[c] < h.cyc_root[bc])) bc = c;
        }
        /* connect every vertex to it: level 0 = its component */
        int32_t left = 0;
        for (int32_t v = 0; v < n; ++v) {
            level[v] = h.cyc[v] == bc ? 0 : -1;
            left += level[v] < 0;
        }
        for (int32_t k = 1; left > 0; ++k) {
            int32_t got = 0;
            for (int32_t v = 0; v < n; ++v) {
                pick[v] = -1;
                if (level[v] >= 0) continue;
                for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
                    int32_t t = col[e];
                    if (level[t] >= 0 && level[t] < k) {
                        pick[v] = e;
                        break;
                    }
                }
            }
            for (int32_t v = 0; v < n; ++v)
                if (pick[v] >= 0) {
                    level[v] = k;
                    h.pi[v] = pick[v];
                    ++got;
                }
            if (got == 0) {
                rc = OR_ERR_NOT_SC;
                goto done;
            }
            left -= got;
        }
        howard_evaluate(&h);   /* one cycle now: values with its lambda */
        bc = 0;
        /* improvement (Jacobi), strict */
        int64_t switched = 0;
        for (int32_t v = 0; v < n; ++v) {
            int32_t best = rp[v];
            for (int32_t e = rp[v] + 1; e < rp[v + 1]; ++e)
                if (howard_better(&h, e, best)) best = e;
            int32_t cur = h.pi[v];
            int sw = howard_key2(&h, best) > howard_key2(&h, cur);
            newpi[v] = sw ? best : cur;
            switched += sw;
        }
        if (switched == 0) break;
        if (++it >= max_iter) {
            rc = OR_ERR_NOT_CONVERGED;
            goto done;
        }
        memcpy(h.pi, newpi, N * sizeof(int32_t));
    }
    if (h.ncyc != 1) {
        rc = OR_ERR_ARG;
        goto done;
    }
    if (num) *num = mode == 0 ? h.cyc_p[0] : -h.cyc_p[0];
    if (den) *den = h.cyc_q[0];
    {
        int32_t r = h.cyc_root[0], x = r, L = 0;
        do {
            if (cycle) cycle[L] = h.pi[x];
            ++L;
            x = h.succ[x];
        } while (x != r);
        if (clen) *clen = L;
    }
    for (int32_t v = 0; v < n; ++v) {
        if (V_out) {
            if (h.V[v] > (i128)INT64_MAX || h.V[v] < (i128)INT64_MIN) {
                rc = OR_ERR_RANGE;
                goto done;
            }
            V_out[v] = (int64_t)h.V[v];
        }
        if (policy) policy[v] = h.pi[v];
    }
    if (iters) *iters = it;
done:
    free(h.pi); free(h.succ); free(h.cyc); free(h.state); free(h.path);
    free(h.S); free(h.T); free(h.V); free(h.cyc_root); free(h.cyc_p); free(h.cyc_q);
    free(newpi); free(level); free(pick);
    return rc;
}

/* Optimal cycle ratio w(C)/t(C) by the same iteration, transit times tt[m] >= 1. */
int oracle_howard_ratio(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                        const int32_t *w, const int32_t *tt, int mode, int64_t max_iter,
                        int64_t *num, int64_t *den, int32_t *cycle, int32_t *clen,
                        int64_t *eta_p, int64_t *eta_q, int64_t *V_out, int32_t *policy,
                        int64_t *iters, const int32_t *init) {
    if (!tt) return OR_ERR_ARG;
    return howard_impl(n, m, rp, col, w, tt, mode, max_iter, num, den, cycle, clen, eta_p,
                       eta_q, V_out, policy, iters, NULL, 0, init);
}

/* ======================================================================== */
/* Karp's recurrence (Karp 1978) with the super-source of Sec. 2.1            */
/* ======================================================================== */
/*
 * Augment G with a new vertex s and 0-weight edges s -> v for all v (Sec. 2.1),
 * N = n + 1 vertices.  D_k(v) = largest weight of a walk of exactly k edges
 * from s to v (-inf if none).  Karp's theorem (max form):
 *     lambda* = max_{v : D_N(v) > -inf}  min_{0 <= k < N, D_k(v) > -inf}
 *                   (D_N(v) - D_k(v)) / (N - k).
 * D_0 is finite only at s, and s has no in-edges, so D_1(v) = 0 for all v and
 * D_k(v) = max over edges (u,v) of D_{k-1}(u) + w for k >= 2.  Two passes keep
 * memory O(n): pass 1 computes D_N, pass 2 recomputes D_1..D_{N-1} and keeps
 * the running minimum per vertex.  Cost 2*N*m.
 */
#define NEG_INF INT64_MIN

static void karp_step(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                      int mode, const int64_t *Dp, int64_t *Dn) {
    for (int32_t v = 0; v < n; ++v) Dn[v] = NEG_INF;
    for (int32_t u = 0; u < n; ++u) {
        if (Dp[u] == NEG_INF) continue;
        for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
            int64_t c = Dp[u] + wmax(w, e, mode);
            if (c > Dn[col[e]]) Dn[col[e]] = c;
        }
    }
}

int oracle_karp(int32_t n, int32_t m, const int32_t *rp, const int32_t *col, const int32_t *w,
                int mode, int64_t *num, int64_t *den) {
    int rc = check_csr(n, m, rp, col);
    if (rc) return rc;
    if (!w || (mode != 0 && mode != 1)) return OR_ERR_ARG;
    for (int32_t e = 0; e < m; ++e)
        if (w[e] == INT32_MIN) return OR_ERR_RANGE;
    int64_t N = (int64_t)n + 1;
    size_t sz = (size_t)n * sizeof(int64_t);
    int64_t *A = malloc(sz), *B = malloc(sz), *DN = malloc(sz), *bp = malloc(sz), *bq = malloc(sz);
    if (!A || !B || !DN || !bp || !bq) {
        free(A); free(B); free(DN); free(bp); free(bq);
        return OR_ERR_NOMEM;
    }
    /* pass 1: D_N */
    for (int32_t v = 0; v < n; ++v) A[v] = 0; /* D_1 */
    for (int64_t k = 2; k <= N; ++k) {
        karp_step(n, rp, col, w, mode, A, B);
        int64_t *t = A; A = B; B = t;
    }
    memcpy(DN, A, sz);
    /* pass 2: min over k = 1..N-1 of (D_N - D_k)/(N - k); D_0(v) = -inf */
    for (int32_t v = 0; v < n; ++v) { bp[v] = 0; bq[v] = 0; } /* bq = 0: unset */
    for (int32_t v = 0; v < n; ++v) A[v] = 0; /* D_1 */
    for (int64_t k = 1; k <= N - 1; ++k) {
        if (k > 1) {
            karp_step(n, rp, col, w, mode, A, B);
            int64_t *t = A; A = B; B = t;
        }
        for (int32_t v = 0; v < n; ++v) {
            if (DN[v] == NEG_INF || A[v] == NEG_INF) continue;
            int64_t p = DN[v] - A[v], q = N - k;
            if (bq[v] == 0 || frac_cmp(p, q, bp[v], bq[v]) < 0) {
                bp[v] = p;
                bq[v] = q;
            }
        }
    }
    int have = 0;
    int64_t P = 0, Q = 1;
    for (int32_t v = 0; v < n; ++v) {
        if (DN[v] == NEG_INF || bq[v] == 0) continue;
        if (!have || frac_cmp(bp[v], bq[v], P, Q) > 0) {
            P = bp[v];
            Q = bq[v];
            have = 1;
        }
    }
    free(A); free(B); free(DN); free(bp); free(bq);
    if (!have) return OR_ERR_ARG;
    int64_t g = gcd64(P, Q);
    P /= g;
    Q /= g;
    if (num) *num = mode == 0 ? P : -P;
    if (den) *den = Q;
    return OR_OK;
}

/* ======================================================================== */
/* Brute force: every simple cycle (tiny graphs)                              */
/* ======================================================================== */
/*
 * Each simple cycle is enumerated once, as the edge sequence that starts at
 * its smallest vertex s: depth-first search from s over vertices > s, every
 * parallel edge a separate branch, closing on any edge back to s.  Returns the
 * best mean (in the given mode) and every cycle attaining it, concatenated in
 * opt_edges with offsets opt_ptr[0..nopt].
 */
typedef struct {
    const int32_t *rp, *col, *w;
    const int32_t *tt;    /* transit times, NULL = 1 per edge */
    int mode;
    int32_t s;
    int32_t *stk_e;
    char *onpath;
    int32_t depth;
    int have;
    int64_t bp, bq;       /* best mean or ratio (max sense) */
    int64_t ncycles;
    int32_t *opt_edges;
    int64_t opt_cap_edges, opt_used_edges;
    int64_t *opt_ptr;
    int64_t opt_cap, nopt;
    int overflow;
} brute_ctx;

static void brute_record(brute_ctx *b, int64_t W, int64_t T, int64_t L) {
    b->ncycles++;
    int c = b->have ? frac_cmp(W, T, b->bp, b->bq) : 1;
    if (c < 0) return;
    if (c > 0) {
        b->have = 1;
        b->bp = W;
        b->bq = T;
        b->nopt = 0;
        b->opt_used_edges = 0;
        b->overflow = 0;
    }
    if (b->nopt >= b->opt_cap || b->opt_used_edges + L > b->opt_cap_edges) {
        b->overflow = 1;
        return;
    }
    b->opt_ptr[b->nopt] = b->opt_used_edges;
    for (int64_t i = 0; i < L; ++i) b->opt_edges[b->opt_used_edges++] = b->stk_e[i];
    b->nopt++;
    b->opt_ptr[b->nopt] = b->opt_used_edges;
}

static void brute_dfs(brute_ctx *b, int32_t u, int64_t W, int64_t T) {
    for (int32_t e = b->rp[u]; e < b->rp[u + 1]; ++e) {
        int32_t t = b->col[e];
        int64_t W2 = W + wmax(b->w, e, b->mode);
        int64_t T2 = T + tval(b->tt, e);
        b->stk_e[b->depth] = e;
        if (t == b->s) {
            brute_record(b, W2, T2, b->depth + 1);
        } else if (t > b->s && !b->onpath[t]) {
            b->onpath[t] = 1;
            b->depth++;
            brute_dfs(b, t, W2, T2);
            b->depth--;
            b->onpath[t] = 0;
        }
    }
}

static int brute_impl(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                      const int32_t *w, const int32_t *tt, int mode, int64_t *num, int64_t *den,
                      int64_t *ncycles, int32_t *opt_edges, int64_t opt_cap_edges,
                      int64_t *opt_ptr, int64_t opt_cap, int64_t *nopt) {
    if (n <= 0 || n > 16 || !rp || !col || !w || (mode != 0 && mode != 1)) return OR_ERR_ARG;
    if (tt)
        for (int32_t e = 0; e < m; ++e)
            if (tt[e] < 1) return OR_ERR_ARG;
    if (rp[0] != 0 || rp[n] != m) return OR_ERR_CSR;
    for (int32_t v = 0; v < n; ++v)
        if (rp[v + 1] < rp[v]) return OR_ERR_CSR;
    for (int32_t e = 0; e < m; ++e)
        if (col[e] < 0 || col[e] >= n || w[e] == INT32_MIN) return OR_ERR_CSR;
    brute_ctx b;
    memset(&b, 0, sizeof b);
    b.rp = rp; b.col = col; b.w = w; b.tt = tt; b.mode = mode;
    int32_t stk[17];
    char onp[16];
    memset(onp, 0, sizeof onp);
    b.stk_e = stk;
    b.onpath = onp;
    b.opt_edges = opt_edges;
    b.opt_cap_edges = opt_cap_edges;
    b.opt_ptr = opt_ptr;
    b.opt_cap = opt_cap;
    if (opt_cap > 0) opt_ptr[0] = 0;
    for (int32_t s = 0; s < n; ++s) {
        b.s = s;
        b.depth = 0;
        onp[s] = 1;
        brute_dfs(&b, s, 0, 0);
        onp[s] = 0;
    }
    if (ncycles) *ncycles = b.ncycles;
    if (!b.have) return OR_ERR_NO_OUT_EDGE; /* acyclic */
    int64_t g = gcd64(b.bp, b.bq);
    if (num) *num = (mode == 0 ? b.bp : -b.bp) / g;
    if (den) *den = b.bq / g;
    if (nopt) *nopt = b.nopt;
    return b.overflow ? OR_ERR_TOO_MANY : OR_OK;
}

int oracle_brute(int32_t n, int32_t m, const int32_t *rp, const int32_t *col, const int32_t *w,
                 int mode, int64_t *num, int64_t *den, int64_t *ncycles, int32_t *opt_edges,
                 int64_t opt_cap_edges, int64_t *opt_ptr, int64_t opt_cap, int64_t *nopt) {
    return brute_impl(n, m, rp, col, w, NULL, mode, num, den, ncycles, opt_edges, opt_cap_edges,
                      opt_ptr, opt_cap, nopt);
}

/* Every simple cycle, best ratio w(C)/t(C) (transit times tt[m] >= 1). */
int oracle_brute_ratio(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                       const int32_t *w, const int32_t *tt, int mode, int64_t *num, int64_t *den,
                       int64_t *ncycles, int32_t *opt_edges, int64_t opt_cap_edges,
                       int64_t *opt_ptr, int64_t opt_cap, int64_t *nopt) {
    if (!tt) return OR_ERR_ARG;
    return brute_impl(n, m, rp, col, w, tt, mode, num, den, ncycles, opt_edges, opt_cap_edges,
                      opt_ptr, opt_cap, nopt);
}

/* ======================================================================== */
/* Tarjan's strongly connected components (iterative)                        */
/* ======================================================================== */
/* comp[v] = component id; ids come out in reverse topological order of the
 * component graph (a sink component first).  Returns the number of
 * components, or a negative code. */
int32_t oracle_tarjan_scc(int32_t n, const int32_t *rp, const int32_t *col, int32_t *comp) {
    if (n <= 0 || !rp || !col || !comp) return OR_ERR_ARG;
    size_t N = (size_t)n;
    int32_t *index = malloc(N * sizeof(int32_t)), *low = malloc(N * sizeof(int32_t));
    int32_t *stk = malloc(N * sizeof(int32_t)), *cs_v = malloc(N * sizeof(int32_t));
    int32_t *cs_e = malloc(N * sizeof(int32_t));
    char *on = calloc(N, 1);
    if (!index || !low || !stk || !cs_v || !cs_e || !on) {
        free(index); free(low); free(stk); free(cs_v); free(cs_e); free(on);
        return OR_ERR_NOMEM;
    }
    for (int32_t v = 0; v < n; ++v) index[v] = -1;
    int32_t next = 0, sp = 0, ncomp = 0;
    for (int32_t r = 0; r < n; ++r) {
        if (index[r] >= 0) continue;
        int32_t csp = 0;
        cs_v[csp] = r; cs_e[csp] = rp[r]; ++csp;
        index[r] = low[r] = next++;
        stk[sp++] = r; on[r] = 1;
        while (csp > 0) {
            int32_t v = cs_v[csp - 1];
            if (cs_e[csp - 1] < rp[v + 1]) {
                int32_t t = col[cs_e[csp - 1]++];
                if (index[t] < 0) {
                    index[t] = low[t] = next++;
                    stk[sp++] = t; on[t] = 1;
                    cs_v[csp] = t; cs_e[csp] = rp[t]; ++csp;
                } else if (on[t] && index[t] < low[v]) {
                    low[v] = index[t];
                }
            } else {
                if (low[v] == index[v]) {
                    int32_t x;
                    do {
                        x = stk[--sp];
                        on[x] = 0;
                        comp[x] = ncomp;
                    } while (x != v);
                    ++ncomp;
                }
                --csp;
                if (csp > 0) {
                    int32_t p = cs_v[csp - 1];
                    if (low[v] < low[p]) low[p] = low[v];
                }
            }
        }
    }
    free(index); free(low); free(stk); free(cs_v); free(cs_e); free(on);
    return ncomp;
}

/* ======================================================================== */
/* Certificate (LP dual of Eq. (1), Prop. 2.1)                               */
/* ======================================================================== */
/*
 * Checks, in the maximising sense (w negated in min mode, num negated too):
 *   (a) every edge e = (v, t): eta(t) <= eta(v)                 [code 1]
 *   (b) if eta(t) = eta(v) = p/q:  q*w(e) - p*t(e) + V(t) - V(v) <= 0
 *       (t(e) = 1 for the mean)                                  [code 2]
 *   (c) the cycle is a closed walk of CSR edges, simple,
 *       and w(C) * den = num * t(C)  (t(C) = |C| for the mean)    [codes 3,4,5]
 *   (d) num/den = max_v eta(v), den > 0                          [code 6]
 * (a)+(b): summing (b) around any cycle (on which eta is constant by (a))
 * shows every cycle mean is <= the eta of its vertices <= max eta; (c)+(d)
 * show that value is attained.  Together: num/den is the optimal mean.
 * Returns 0 if all hold, else the code of the first failure; *bad receives
 * the offending edge or vertex index.
 */
static int certificate_impl(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                            const int32_t *w, const int32_t *tt, int mode, const int64_t *eta_p,
                            const int64_t *eta_q, const int64_t *V, int64_t num, int64_t den,
                            const int32_t *cycle, int32_t clen, int64_t *bad) {
    if (check_csr(n, m, rp, col)) return -1;
    if (mode != 0 && mode != 1) return -1;
    int64_t P = mode == 0 ? num : -num;
    if (den <= 0) return 6;
    for (int32_t v = 0; v < n; ++v) {
        if (eta_q[v] <= 0) { if (bad) *bad = v; return 1; }
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
            int32_t t = col[e];
            int c = frac_cmp(eta_p[t], eta_q[t], eta_p[v], eta_q[v]);
            if (c > 0) { if (bad) *bad = e; return 1; }
            if (c == 0) {
                i128 red = (i128)eta_q[v] * wmax(w, e, mode) - (i128)eta_p[v] * tval(tt, e) +
                           V[t] - V[v];
                if (red > 0) { if (bad) *bad = e; return 2; }
            }
        }
    }
    if (clen <= 0 || clen > n) return 3;
    char *seen = calloc((size_t)n, 1);
    if (!seen) return -1;
    /* source of each cycle edge: binary search in rp */
    int32_t first_src = -1, prev_t = -1;
    i128 W = 0, Tc = 0;
    int code = 0;
    int32_t i = 0;
    for (i = 0; i < clen && !code; ++i) {
        int32_t e = cycle[i];
        if (e < 0 || e >= m) { code = 3; break; }
        int32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            int32_t mid = lo + (hi - lo + 1) / 2;
            if (rp[mid] <= e) lo = mid; else hi = mid - 1;
        }
        int32_t src = lo;
        if (i == 0) first_src = src;
        else if (src != prev_t) { code = 3; break; }
        if (seen[src]) { code = 4; break; }
        seen[src] = 1;
        prev_t = col[e];
        W += wmax(w, e, mode);
        Tc += tval(tt, e);
    }
    free(seen);
    if (code) { if (bad) *bad = i; return code; }
    if (prev_t != first_src) return 3;
    if (W * den != (i128)P * Tc) return 5;
    /* (d) */
    int32_t arg = 0;
    for (int32_t v = 1; v < n; ++v)
        if (frac_cmp(eta_p[v], eta_q[v], eta_p[arg], eta_q[arg]) > 0) arg = v;
    if (frac_cmp(eta_p[arg], eta_q[arg], P, den) != 0) { if (bad) *bad = arg; return 6; }
    return 0;
}

int oracle_certificate(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                       const int32_t *w, int mode, const int64_t *eta_p, const int64_t *eta_q,
                       const int64_t *V, int64_t num, int64_t den, const int32_t *cycle,
                       int32_t clen, int64_t *bad) {
    return certificate_impl(n, m, rp, col, w, NULL, mode, eta_p, eta_q, V, num, den, cycle,
                            clen, bad);
}

/* The same check for an optimal cycle ratio (transit times tt[m] >= 1). */
int oracle_certificate_ratio(int32_t n, int32_t m, const int32_t *rp, const int32_t *col,
                             const int32_t *w, const int32_t *tt, int mode,
                             const int64_t *eta_p, const int64_t *eta_q, const int64_t *V,
                             int64_t num, int64_t den, const int32_t *cycle, int32_t clen,
                             int64_t *bad) {
    if (!tt) return -1;
    return certificate_impl(n, m, rp, col, w, tt, mode, eta_p, eta_q, V, num, den, cycle, clen,
                            bad);
}

