/*
 * synth.c -- seeded synthetic graph generators for the optimal-cycle-mean
 * workloads.
 *
 * This module only builds inputs: CSR digraphs (row_ptr, col_idx, w) with
 * int32 weights.  It contains none of the cycle-mean arithmetic, so both the
 * CPU oracle and the CUDA solver can be fed from it.
 *
 * Determinism: every random number comes from a counter-based SplitMix64
 * stream keyed by (seed, tag, index), bounded integers use Lemire's unbiased
 * multiply-and-reject method, and nothing uses floating point or libm.  The
 * same seed therefore gives the same bytes on x86_64 and aarch64, in any
 * thread count.
 *
 * Workload families (the paper's DiVinE state spaces, road and DIMACS graphs
 * are not available; these stand in for them, see the experimental section
 * of the paper, Sec. 4):
 *   ring_extra   : ring i -> i+1 (mod n) plus U{xlo..xhi} extra edges per
 *                  vertex with uniform targets; weights wscale*U[wlo,whi].
 *   product      : synchronous-interleaving product of P local processes,
 *                  each an S-state ring with C random chords per state;
 *                  vertices numbered in BFS order from the all-zero state
 *                  (a model-checker state space, Sec. 2.2 / Sec. 4).
 *   locality     : out-degree 4/16/64 mix, ring edge first, other targets
 *                  i + 1 + floor(|X|) (mod n), X ~ N(0, sigma) by Irwin-Hall.
 *   batch sizes  : log-uniform vertex counts, integer fixed-point exp2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } sm64;

static inline uint64_t fmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t sm64_next(sm64 *g) {
    g->s += 0x9E3779B97F4A7C15ULL;
    return fmix64(g->s);
}

/* Independent stream for (seed, tag, idx). */
static inline sm64 stream(uint64_t seed, uint64_t tag, uint64_t idx) {
    sm64 g;
    uint64_t a = fmix64(seed + 0x9E3779B97F4A7C15ULL);
    uint64_t b = fmix64(a ^ (tag * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL));
    g.s = fmix64(b ^ (idx * 0xAEF17502108EF2D9ULL + 0x632BE59BD9B4E019ULL));
    return g;
}

/* Uniform integer in [0, range), range >= 1 (Lemire 2019, unbiased). */
static inline uint32_t bounded(sm64 *g, uint32_t range) {
    uint32_t x = (uint32_t)(sm64_next(g) >> 32);
    uint64_t m = (uint64_t)x * (uint64_t)range;
    uint32_t l = (uint32_t)m;
    if (l < range) {
        uint32_t t = (uint32_t)(0u - range) % range;
        while (l < t) {
            x = (uint32_t)(sm64_next(g) >> 32);
            m = (uint64_t)x * (uint64_t)range;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

/* Uniform integer in [lo, hi] inclusive. */
static inline int64_t uniform_incl(sm64 *g, int64_t lo, int64_t hi) {
    return lo + (int64_t)bounded(g, (uint32_t)(hi - lo + 1));
}

/* ------------------------------------------------------------------------ */
/* ring_extra family                                                         */
/* ------------------------------------------------------------------------ */
/* Per vertex i (stream (seed, tag, i)): draw k = U{xlo..xhi}; the row is the
 * ring edge i -> (i+1) mod n followed by k edges with targets U[0,n); then one
 * weight per edge in row order, wscale * U[wlo, whi]. */

int synth_ring_extra_degrees(uint64_t seed, uint64_t tag, int32_t n, int32_t xlo,
                             int32_t xhi, int32_t *deg_out) {
    if (n <= 0 || xlo < 0 || xhi < xlo) return -1;
    for (int32_t i = 0; i < n; ++i) {
        sm64 g = stream(seed, tag, (uint64_t)i);
        deg_out[i] = 1 + (int32_t)uniform_incl(&g, xlo, xhi);
    }
    return 0;
}

int synth_ring_extra_fill(uint64_t seed, uint64_t tag, int32_t n, int32_t xlo, int32_t xhi,
                          int32_t wlo, int32_t whi, int32_t wscale, const int32_t *row_ptr,
                          int32_t *col, int32_t *w) {
    if (n <= 0 || xlo < 0 || xhi < xlo || whi < wlo) return -1;
    for (int32_t i = 0; i < n; ++i) {
        sm64 g = stream(seed, tag, (uint64_t)i);
        int32_t k = (int32_t)uniform_incl(&g, xlo, xhi);
        int32_t e = row_ptr[i];
        if (row_ptr[i + 1] - e != k + 1) return -2;
        col[e] = (i + 1 == n) ? 0 : i + 1;
        for (int32_t j = 1; j <= k; ++j) col[e + j] = (int32_t)bounded(&g, (uint32_t)n);
        for (int32_t j = 0; j <= k; ++j)
            w[e + j] = (int32_t)(wscale * uniform_incl(&g, wlo, whi));
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* locality family                                                           */
/* ------------------------------------------------------------------------ */
/* Per vertex i (stream (seed, tag, i)): u = U[0,30): deg 64 if u == 0,
 * deg 16 if 1 <= u <= 5, else deg 4 (mean 8).  Row: ring edge first, then
 * deg-1 edges; each non-ring edge draws three 64-bit words = twelve 16-bit
 * uniforms u_j, X*sigma_scale = (sum u_j - 6*65536) * sigma / 65536, and the
 * offset is 1 + floor(|X|).  Then one weight per edge in row order, U[wlo,whi]. */

static inline int32_t locality_degree(sm64 *g) {
    uint32_t u = bounded(g, 30);
    return u == 0 ? 64 : (u <= 5 ? 16 : 4);
}

int synth_locality_degrees(uint64_t seed, uint64_t tag, int32_t n, int32_t *deg_out) {
    if (n <= 1) return -1;
    for (int32_t i = 0; i < n; ++i) {
        sm64 g = stream(seed, tag, (uint64_t)i);
        deg_out[i] = locality_degree(&g);
    }
    return 0;
}

int synth_locality_fill(uint64_t seed, uint64_t tag, int32_t n, int32_t sigma, int32_t wlo,
                        int32_t whi, const int32_t *row_ptr, int32_t *col, int32_t *w) {
    if (n <= 1 || sigma <= 0 || whi < wlo) return -1;
    for (int32_t i = 0; i < n; ++i) {
        sm64 g = stream(seed, tag, (uint64_t)i);
        int32_t d = locality_degree(&g);
        int32_t e = row_ptr[i];
        if (row_ptr[i + 1] - e != d) return -2;
        col[e] = (i + 1 == n) ? 0 : i + 1;
        for (int32_t j = 1; j < d; ++j) {
            int64_t sum = 0;
            for (int r = 0; r < 3; ++r) {
                uint64_t x = sm64_next(&g);
                sum += (int64_t)(x & 0xFFFF) + (int64_t)((x >> 16) & 0xFFFF) +
                       (int64_t)((x >> 32) & 0xFFFF) + (int64_t)(x >> 48);
            }
            int64_t dev = sum - 6 * 65536;
            if (dev < 0) dev = -dev;
            int64_t off = 1 + ((dev * (int64_t)sigma) >> 16);
            col[e + j] = (int32_t)(((int64_t)i + off) % (int64_t)n);
        }
        for (int32_t j = 0; j < d; ++j) w[e + j] = (int32_t)uniform_incl(&g, wlo, whi);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* product (state-space) family                                              */
/* ------------------------------------------------------------------------ */
/* P processes (P <= 8), each with S local states (S^P <= 2^31 - 1).  Process p,
 * state s (stream (seed, tag + 1 + p, s)): local moves are the ring move
 * s -> (s+1) mod S, then C chord targets U[0,S), dropping a chord equal to s or
 * to an earlier move of s.  A global state moves by one local move of one
 * process (interleaving).  Vertices are numbered in BFS order from the all-zero
 * state, successors visited for p = 0..P-1 and each process's moves in order;
 * a row lists the successors in that order.  Weights: stream (seed, tag, id),
 * one U[wlo,whi] per row slot. */

typedef struct {
    int32_t P, S, C;
    int32_t *ldeg;   /* [P*S] */
    int32_t *lmov;   /* [P*S*(C+1)] */
} product_spec;

static int product_build_local(uint64_t seed, uint64_t tag, product_spec *ps) {
    int32_t P = ps->P, S = ps->S, C = ps->C;
    ps->ldeg = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * S);
    ps->lmov = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * S * (C + 1));
    if (!ps->ldeg || !ps->lmov) return -3;
    for (int32_t p = 0; p < P; ++p) {
        for (int32_t s = 0; s < S; ++s) {
            sm64 g = stream(seed, tag + 1 + (uint64_t)p, (uint64_t)s);
            int32_t *mv = ps->lmov + ((size_t)p * S + s) * (C + 1);
            int32_t k = 0;
            mv[k++] = (s + 1) % S;
            for (int32_t c = 0; c < C; ++c) {
                int32_t t = (int32_t)bounded(&g, (uint32_t)S);
                int dup = (t == s);
                for (int32_t j = 0; j < k && !dup; ++j) dup = (mv[j] == t);
                if (!dup) mv[k++] = t;
            }
            ps->ldeg[(size_t)p * S + s] = k;
        }
    }
    return 0;
}

static void product_free(product_spec *ps) {
    free(ps->ldeg);
    free(ps->lmov);
}

/* Number of global states S^P, or -1 when out of range. */
int64_t synth_product_num_states(int32_t P, int32_t S) {
    if (P < 1 || P > 8 || S < 2) return -1;
    int64_t N = 1;
    for (int32_t p = 0; p < P; ++p) {
        N *= S;
        if (N > 0x7FFFFFFFLL) return -1;
    }
    return N;
}

/* Fills deg_out[N] (row lengths in BFS numbering) and perm_out[N]: the
 * mixed-radix code (s_0 + S*s_1 + ...) of the state with BFS id i. */
int synth_product_structure(uint64_t seed, uint64_t tag, int32_t P, int32_t S, int32_t C,
                            int32_t *deg_out, int32_t *code_of_id) {
    int64_t N = synth_product_num_states(P, S);
    if (N < 0 || C < 0) return -1;
    product_spec ps = {P, S, C, NULL, NULL};
    if (product_build_local(seed, tag, &ps)) { product_free(&ps); return -3; }
    int32_t *id_of_code = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!id_of_code) { product_free(&ps); return -3; }
    for (int64_t i = 0; i < N; ++i) id_of_code[i] = -1;
    int64_t pw[8];
    pw[0] = 1;
    for (int32_t p = 1; p < P; ++p) pw[p] = pw[p - 1] * S;
    int64_t head = 0, tail = 0;
    code_of_id[tail++] = 0;
    id_of_code[0] = 0;
    while (head < tail) {
        int32_t code = code_of_id[head];
        int32_t d = 0;
        for (int32_t p = 0; p < P; ++p) {
            int32_t sp = (int32_t)((code / pw[p]) % S);
            const int32_t *mv = ps.lmov + ((size_t)p * S + sp) * (C + 1);
            int32_t k = ps.ldeg[(size_t)p * S + sp];
            for (int32_t j = 0; j < k; ++j) {
                int32_t nc = (int32_t)(code + (mv[j] - sp) * pw[p]);
                if (id_of_code[nc] < 0) {
                    id_of_code[nc] = (int32_t)tail;
                    code_of_id[tail++] = nc;
                }
                ++d;
            }
        }
        deg_out[head] = d;
        ++head;
    }
    free(id_of_code);
    product_free(&ps);
    return tail == N ? 0 : -4;
}

int synth_product_fill(uint64_t seed, uint64_t tag, int32_t P, int32_t S, int32_t C,
                       int32_t wlo, int32_t whi, const int32_t *code_of_id,
                       const int32_t *row_ptr, int32_t *col, int32_t *w) {
    int64_t N = synth_product_num_states(P, S);
    if (N < 0 || C < 0 || whi < wlo) return -1;
    product_spec ps = {P, S, C, NULL, NULL};
    if (product_build_local(seed, tag, &ps)) { product_free(&ps); return -3; }
    int32_t *id_of_code = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!id_of_code) { product_free(&ps); return -3; }
    for (int64_t i = 0; i < N; ++i) id_of_code[code_of_id[i]] = (int32_t)i;
    int64_t pw[8];
    pw[0] = 1;
    for (int32_t p = 1; p < P; ++p) pw[p] = pw[p - 1] * S;
    for (int64_t i = 0; i < N; ++i) {
        int32_t code = code_of_id[i];
        int32_t e = row_ptr[i];
        for (int32_t p = 0; p < P; ++p) {
            int32_t sp = (int32_t)((code / pw[p]) % S);
            const int32_t *mv = ps.lmov + ((size_t)p * S + sp) * (C + 1);
            int32_t k = ps.ldeg[(size_t)p * S + sp];
            for (int32_t j = 0; j < k; ++j)
                col[e++] = id_of_code[(int32_t)(code + (mv[j] - sp) * pw[p])];
        }
        if (e != row_ptr[i + 1]) { free(id_of_code); product_free(&ps); return -2; }
        sm64 g = stream(seed, tag, (uint64_t)i);
        for (int32_t f = row_ptr[i]; f < e; ++f) w[f] = (int32_t)uniform_incl(&g, wlo, whi);
    }
    free(id_of_code);
    product_free(&ps);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* log-uniform sizes for the batched workload                               */
/* ------------------------------------------------------------------------ */
/* n_g = floor(nmin * (nmax/nmin)^u), u = U32/2^32, in integer fixed point:
 * log2(ratio) by the bit-by-bit squaring method (Q58), 2^f by the exp Taylor
 * series of f*ln2 (Q62).  Bit-identical on every platform. */

typedef unsigned __int128 u128;

static uint64_t log2_q58(uint64_t x) { /* x >= 1 */
    int ip = 63 - __builtin_clzll(x);
    /* y = x / 2^ip in Q62, in [1, 2) */
    u128 y = ((u128)x << 62) >> ip;
    uint64_t frac = 0;
    for (int b = 57; b >= 0; --b) {
        y = (y * y) >> 62;
        if (y >= ((u128)2 << 62)) {
            frac |= (uint64_t)1 << b;
            y >>= 1;
        }
    }
    return ((uint64_t)ip << 58) | frac;
}

static const uint64_t LN2_Q62 = 3196577161300663914ULL;

static uint64_t exp2_frac_q62(uint64_t f_q58) { /* 2^f for f in [0,1), result Q62 */
    u128 x = ((u128)f_q58 * LN2_Q62) >> 58;    /* f*ln2, Q62 */
    u128 term = (u128)1 << 62, sum = term;
    for (uint64_t k = 1; k < 40 && term != 0; ++k) {
        term = (term * x) >> 62;
        term /= k;
        sum += term;
    }
    return (uint64_t)sum;
}

int synth_loguniform_sizes(uint64_t seed, uint64_t tag, int32_t G, int32_t nmin, int32_t nmax,
                           int32_t *sizes) {
    if (G <= 0 || nmin < 1 || nmax < nmin) return -1;
    uint64_t ratio_num = (uint64_t)nmax, ratio_den = (uint64_t)nmin;
    /* log2(nmax/nmin) = log2(nmax) - log2(nmin) in Q58 */
    uint64_t L = log2_q58(ratio_num) - log2_q58(ratio_den);
    for (int32_t g = 0; g < G; ++g) {
        sm64 s = stream(seed, tag, (uint64_t)g);
        uint64_t u = sm64_next(&s) >> 32;                 /* Q32 in [0,1) */
        uint64_t y = (uint64_t)(((u128)u * L) >> 32);     /* Q58 */
        uint64_t ip = y >> 58, fr = y & ((1ULL << 58) - 1);
        uint64_t e = exp2_frac_q62(fr);                   /* Q62 */
        u128 v = ((u128)nmin * e) << ip;                  /* Q62 */
        int64_t ng = (int64_t)(v >> 62);
        if (ng < nmin) ng = nmin;
        if (ng > nmax) ng = nmax;
        sizes[g] = (int32_t)ng;
    }
    return 0;
}

/* Cheap 64-bit digest of an int32 array (for fixture checks). */
uint64_t synth_digest_i32(const int32_t *a, int64_t len) {
    uint64_t h = 0x243F6A8885A308D3ULL;
    for (int64_t i = 0; i < len; ++i) h = fmix64(h ^ (uint64_t)(uint32_t)a[i]) + (uint64_t)i;
    return h;
}
