/*
 * rw_oracle.c -- CPU oracle for the random-walk incomplete LDL^T preconditioner.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may call it.  Plain loops in the order
 * the paper describes the method; nothing blocked, fused or reordered.  Built
 * with -ffp-contract=off so that every floating-point operation below is one
 * IEEE-rounded operation (no fused multiply-add).
 *
 * Paper: H. Qian, S. S. Sapatnekar, "Stochastic Preconditioning for Iterative
 * Linear Equation Solvers".  Citations name the paper's sections and equations.
 */
#include "rw_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10, from its published definition (Salmon et al., SC'11):      */
/* each round multiplies words 0 and 2 by fixed constants, swaps the halves   */
/* and xors in the round key; the key is bumped by two Weyl constants.        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

uint32_t orc_draw(uint64_t seed, uint32_t matrix_index, uint32_t tag, uint32_t k,
                  uint32_t w, uint64_t s) {
    uint32_t ctr[4] = {(uint32_t)(s / 4), w, k, (matrix_index << 2) | (tag & 3u)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[s % 4];
}

/* ------------------------------------------------------------------------ */
/* Transition probabilities of the walk game (Sec. 2.1, Eq. map): from node l */
/* the walker moves to j with probability -A_lj / A_ll and is absorbed at     */
/* ground with the remaining probability (the diagonal excess).  Sampling     */
/* rule: with cumulative weight c_m over the off-diagonal entries in ascending */
/* column order, threshold t_m = min(2^32 - 1, floor(2^32 * (c_m / A_ll)));   */
/* a 32-bit draw u selects the least m with u < t_m, and ground if none.      */
/* ------------------------------------------------------------------------ */
static uint32_t to_threshold(double x) {
    double s = x * 4294967296.0;       /* exact: scaling by a power of two */
    if (!(s < 4294967295.0)) return 0xFFFFFFFFu;
    return (uint32_t)s;                /* truncation = floor for s >= 0 */
}

static int32_t diag_pos(const int32_t* rowptr, const int32_t* col, int32_t l) {
    for (int32_t p = rowptr[l]; p < rowptr[l + 1]; ++p)
        if (col[p] == l) return p;
    return -1;
}

int32_t orc_row_thresholds(const int32_t* rowptr, const int32_t* col, const double* val,
                           int32_t l, uint32_t* t_out) {
    int32_t dp = diag_pos(rowptr, col, l);
    double all = val[dp];
    double c = 0.0;
    int32_t m = 0;
    for (int32_t p = rowptr[l]; p < rowptr[l + 1]; ++p) {
        if (p == dp) continue;
        c = c + (-val[p]);
        t_out[m++] = to_threshold(c / all);
    }
    return m;
}

/* Per-node tables built once per matrix: off-diagonal columns and thresholds
 * in CSR order (diagonal removed), and the first-step table of each row over
 * its upper neighbours j > k (Sec. 5.2). */
typedef struct {
    int32_t n;
    int32_t* off;      /* [n+1] start of node l's off-diagonal entries */
    int32_t* nbr;      /* neighbour column */
    uint32_t* thr;     /* full transition thresholds */
    int32_t* up0;      /* [n] index (into nbr) of the first upper neighbour */
    uint32_t* fthr;    /* first-step thresholds, same indexing as nbr (upper part only) */
    double* S;         /* [n] S_k = sum_{j>k} A_kj (sequential, ascending columns) */
    double* diag;      /* [n] A_kk */
} tables;

static void tables_free(tables* t) {
    free(t->off); free(t->nbr); free(t->thr); free(t->up0); free(t->fthr);
    free(t->S); free(t->diag);
}

static int tables_build(int32_t n, const int32_t* rowptr, const int32_t* col,
                        const double* val, tables* t) {
    int64_t nnz = rowptr[n];
    memset(t, 0, sizeof(*t));
    t->n = n;
    t->off = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
    t->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    t->thr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nnz > 0 ? nnz : 1));
    t->fthr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nnz > 0 ? nnz : 1));
    t->up0 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    t->S = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    t->diag = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!t->off || !t->nbr || !t->thr || !t->fthr || !t->up0 || !t->S || !t->diag) {
        tables_free(t);
        return -4;
    }
    int32_t q = 0;
    for (int32_t l = 0; l < n; ++l) {
        t->off[l] = q;
        int32_t dp = diag_pos(rowptr, col, l);
        t->diag[l] = val[dp];
        int32_t m = orc_row_thresholds(rowptr, col, val, l, t->thr + q);
        int32_t up = -1;
        for (int32_t p = rowptr[l], i = 0; p < rowptr[l + 1]; ++p) {
            if (p == dp) continue;
            t->nbr[q + i] = col[p];
            if (up < 0 && col[p] > l) up = q + i;
            ++i;
        }
        t->up0[l] = up;
        /* First step among the upper neighbours only, probability proportional
         * to -A_kj (Sec. 5.2): cumulative cu_m over j > k, threshold of
         * cu_m / cu_last.  S_k = -cu_last. */
        double cu = 0.0;
        if (up >= 0) {
            for (int32_t p = rowptr[l]; p < rowptr[l + 1]; ++p)
                if (col[p] > l) cu = cu + (-val[p]);
            double c = 0.0;
            int32_t i = up;
            for (int32_t p = rowptr[l]; p < rowptr[l + 1]; ++p) {
                if (col[p] <= l) continue;
                c = c + (-val[p]);
                t->fthr[i++] = to_threshold(c / cu);
            }
        }
        t->S[l] = -cu;
        q += m;
    }
    t->off[n] = q;
    return 0;
}

int orc_validate(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val) {
    if (n < 0 || rowptr[0] != 0) return -2;
    for (int32_t l = 0; l < n; ++l) {
        if (rowptr[l + 1] < rowptr[l]) return -2;
        int has_diag = 0;
        double sum = 0.0, dg = 0.0;
        for (int32_t p = rowptr[l]; p < rowptr[l + 1]; ++p) {
            if (col[p] < 0 || col[p] >= n) return -2;
            if (p > rowptr[l] && col[p] <= col[p - 1]) return -2;
            if (col[p] == l) {
                has_diag = 1;
                dg = val[p];
                if (!(val[p] > 0.0) || !isfinite(val[p])) return -2;
            } else {
                if (!(val[p] < 0.0) || !isfinite(val[p])) return -2;
                sum = sum + (-val[p]);
            }
        }
        if (!has_diag) return -2;
        if (dg - sum < -1e-12 * dg) return -2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Journey record and factor                                                  */
/* ------------------------------------------------------------------------ */
struct orc_factor {
    int32_t n;
    int64_t nnz, cap;
    int64_t* rowptr;
    int32_t* col;
    double* val;
    double* D;
    uint64_t *M, *J, *G, *hops;
};

static int factor_push(orc_factor* f, int32_t c, double v) {
    if (f->nnz == f->cap) {
        int64_t nc = f->cap ? 2 * f->cap : 1024;
        int32_t* nc_col = (int32_t*)realloc(f->col, sizeof(int32_t) * (size_t)nc);
        if (!nc_col) return -4;
        f->col = nc_col;
        double* nc_val = (double*)realloc(f->val, sizeof(double) * (size_t)nc);
        if (!nc_val) return -4;
        f->val = nc_val;
        f->cap = nc;
    }
    f->col[f->nnz] = c;
    f->val[f->nnz] = v;
    f->nnz++;
    return 0;
}

void orc_factor_free(orc_factor* f) {
    if (!f) return;
    free(f->rowptr); free(f->col); free(f->val); free(f->D);
    free(f->M); free(f->J); free(f->G); free(f->hops);
    free(f);
}

int64_t orc_factor_nnz(const orc_factor* f) { return f->nnz; }

void orc_factor_get(const orc_factor* f, int64_t* rowptr, int32_t* col, double* val, double* D,
                    uint64_t* M, uint64_t* J, uint64_t* G, uint64_t* hops) {
    size_t n = (size_t)f->n;
    if (rowptr) memcpy(rowptr, f->rowptr, sizeof(int64_t) * (n + 1));
    if (col) memcpy(col, f->col, sizeof(int32_t) * (size_t)f->nnz);
    if (val) memcpy(val, f->val, sizeof(double) * (size_t)f->nnz);
    if (D) memcpy(D, f->D, sizeof(double) * n);
    if (M) memcpy(M, f->M, sizeof(uint64_t) * n);
    if (J) memcpy(J, f->J, sizeof(uint64_t) * n);
    if (G) memcpy(G, f->G, sizeof(uint64_t) * n);
    if (hops) memcpy(hops, f->hops, sizeof(uint64_t) * n);
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Sampling helpers (the rule stated above tables_build). */
static int32_t sample_full(const tables* t, int32_t l, uint32_t u) {
    int32_t deg = t->off[l + 1] - t->off[l];
    for (int32_t m = 0; m < deg; ++m)
        if (u < t->thr[t->off[l] + m]) return m;
    return -1; /* ground */
}

static int32_t sample_first(const tables* t, int32_t k, uint32_t u) {
    int32_t first = t->up0[k], last = t->off[k + 1];
    for (int32_t i = first; i < last; ++i)
        if (u < t->fthr[i]) return t->nbr[i];
    return t->nbr[last - 1];
}

/* Counters of the journey record for the row being processed:
 * cnt[i] = H'_{k,i}, with the list of touched i. */
typedef struct {
    uint64_t* cnt_all;   /* [n] H' counts of the current row (mode 0) */
    int32_t* touched;
    int32_t ntouched;
} rowacc;

/*
 * One walk from row k (Sec. 3.1 with the one-step-exact first step of Sec.
 * 5.2).  Rows 0..k-1 are homes, ground absorbs.  Step h (h = 1, 2, ...) uses
 * draw number h-1.  A walk that has made max_steps hops without ending is an
 * error.  Returns 0, or -3 on the step cap.  *end = home node, or -1 (ground).
 */
static int one_walk(const tables* t, uint64_t seed, uint32_t mi, uint32_t tag, int32_t k,
                    uint32_t w, uint64_t max_steps, int32_t* end, uint32_t* returns,
                    uint64_t* hops, int32_t* path, int64_t path_cap, int64_t* path_len) {
    uint32_t ret = 0;
    uint64_t h = 1;
    int32_t cur = sample_first(t, k, orc_draw(seed, mi, tag, (uint32_t)k, w, 0));
    if (path) { path[0] = k; path[1] = cur; *path_len = 2; }
    for (;;) {
        if (h >= max_steps) { *hops = h; return -3; }
        uint32_t u = orc_draw(seed, mi, tag, (uint32_t)k, w, h);
        h = h + 1;
        int32_t m = sample_full(t, cur, u);
        int32_t nxt = (m < 0) ? -1 : t->nbr[t->off[cur] + m];
        if (path) {
            if (*path_len >= path_cap) return -4;
            path[(*path_len)++] = nxt;
        }
        if (m < 0) { *end = -1; break; }
        if (nxt < k) { *end = nxt; break; }
        if (nxt == k) ret++;
        cur = nxt;
    }
    *returns = ret;
    *hops = h;
    return 0;
}

/* Algorithm 2 applied to one simulated walk (Sec. 5.3).  path[0..len) are the
 * visited nodes, path[len-1] is the home or ground (-1, taken as a virtual node
 * below every row).  Extracted legal sub-walks of at least two steps add one
 * walk to M of their start node, one visit to J of their start node and, when
 * they end at a node (not ground), one count to H; G counts ground ends.
 * Returns through the callback arrays.  Positions are 0-based here. */
typedef struct {
    int32_t* node;
    int64_t* pos;
    int64_t cap;
} stacks;

typedef struct {
    uint64_t *M, *J, *G;
    /* H updates are appended as (start, end) pairs */
    int32_t* hs; int32_t* he; int64_t nh, hcap;
} reuse_out;

static int reuse_push_h(reuse_out* o, int32_t s, int32_t e) {
    if (o->nh == o->hcap) {
        int64_t nc = o->hcap ? 2 * o->hcap : 4096;
        int32_t* a = (int32_t*)realloc(o->hs, sizeof(int32_t) * (size_t)nc);
        if (!a) return -4;
        o->hs = a;
        int32_t* b = (int32_t*)realloc(o->he, sizeof(int32_t) * (size_t)nc);
        if (!b) return -4;
        o->he = b;
        o->hcap = nc;
    }
    o->hs[o->nh] = s; o->he[o->nh] = e; o->nh++;
    return 0;
}

static int reuse_walk(const int32_t* path, int64_t len, stacks* st, reuse_out* o) {
    int64_t top = 0;
    st->node[0] = path[0];
    st->pos[0] = 0;
    for (int64_t l = 1; l < len; ++l) {
        int32_t kl = path[l];
        while (top >= 0 && kl < st->node[top]) {
            if (l > st->pos[top] + 1) {
                int32_t kp = st->node[top];
                o->M[kp] += 1;
                o->J[kp] += 1;
                if (kl >= 0) { if (reuse_push_h(o, kp, kl)) return -4; }
                else o->G[kp] += 1;
            }
            --top;
        }
        if (top < 0) break;
        if (kl > st->node[top]) {
            ++top;
            if (top >= st->cap) return -4;
            st->node[top] = kl;
            st->pos[top] = l;
        } else {
            o->J[kl] += 1;
        }
    }
    return 0;
}

int32_t orc_reuse_trace(const int32_t* seq, int32_t len, int32_t nlabels,
                        int64_t* dM, int64_t* dJ, int32_t* hs, int32_t* he, int32_t cap) {
    uint64_t* M = (uint64_t*)calloc((size_t)nlabels + 1, sizeof(uint64_t));
    uint64_t* J = (uint64_t*)calloc((size_t)nlabels + 1, sizeof(uint64_t));
    uint64_t* G = (uint64_t*)calloc((size_t)nlabels + 1, sizeof(uint64_t));
    stacks st = {(int32_t*)malloc(sizeof(int32_t) * (size_t)len),
                 (int64_t*)malloc(sizeof(int64_t) * (size_t)len), len};
    reuse_out o = {M, J, G, NULL, NULL, 0, 0};
    int32_t rc = reuse_walk(seq, len, &st, &o);
    if (rc == 0) {
        for (int32_t i = 0; i <= nlabels; ++i) { dM[i] += (int64_t)M[i]; dJ[i] += (int64_t)J[i]; }
        for (int64_t i = 0; i < o.nh && i < cap; ++i) { hs[i] = o.hs[i]; he[i] = o.he[i]; }
        rc = (int32_t)o.nh;
    }
    free(M); free(J); free(G); free(st.node); free(st.pos); free(o.hs); free(o.he);
    return rc;
}

/* One row of Y and D from the counters (Sec. 5.2, Eqs. newy and newz; D from
 * Eq. d as D_kk = 1 / Z_kk):
 *   a    = S_k / A_kk,   S_k = sum_{j>k} A_kj
 *   Y_ki = A_ki / A_kk + a * H'_ki / M'_k           (A_ki = 0 if i is not a neighbour)
 *   D_kk = A_kk / (1 + a * (1 - J'_k / M'_k))
 * Rows without an upper neighbour are exact and use no walks:
 *   Y_ki = A_ki / A_kk, D_kk = A_kk.
 * Entries with |Y_ki| < drop_tol are dropped (the post-processing drop of the
 * footnote in Sec. 4, threshold reading). */
static int emit_row(orc_factor* f, const int32_t* rowptr, const int32_t* col, const double* val,
                    const tables* t, int32_t k, uint64_t* cnt, int32_t* list,
                    int32_t nlist, double drop_tol) {
    double akk = t->diag[k];
    int walked = t->up0[k] >= 0;
    if (!walked) {
        for (int32_t p = rowptr[k]; p < rowptr[k + 1] && col[p] < k; ++p) {
            double y = val[p] / akk;
            if (fabs(y) >= drop_tol) { if (factor_push(f, col[p], y)) return -4; }
        }
        f->D[k] = akk;
        return 0;
    }
    double a = t->S[k] / akk;
    double Mk = (double)f->M[k];
    /* union of the lower neighbours of k and the end nodes, ascending */
    int32_t nl = nlist;
    for (int32_t p = rowptr[k]; p < rowptr[k + 1] && col[p] < k; ++p)
        if (cnt[col[p]] == 0) list[nl++] = col[p];
    qsort(list, (size_t)nl, sizeof(int32_t), cmp_i32);
    int32_t p = rowptr[k];
    for (int32_t s = 0; s < nl; ++s) {
        int32_t i = list[s];
        while (p < rowptr[k + 1] && col[p] < i) ++p;
        double d = (p < rowptr[k + 1] && col[p] == i) ? val[p] / akk : 0.0;
        double r = (double)cnt[i] / Mk;
        double y = d + a * r;
        if (fabs(y) >= drop_tol) { if (factor_push(f, i, y)) return -4; }
    }
    for (int32_t s = 0; s < nl; ++s) cnt[list[s]] = 0; /* clear this row's H' counts */
    double q = (double)f->J[k] / Mk;
    f->D[k] = akk / (1.0 + a * (1.0 - q));
    return 0;
}

int orc_factor_build(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const uint32_t* budget, uint64_t seed, uint32_t matrix_index, uint32_t tag,
                     double drop_tol, uint64_t max_steps, int32_t mode,
                     const int32_t* rows, int32_t nrows,
                     int32_t* rec_end, uint32_t* rec_ret, uint32_t* rec_len, int64_t rec_cap,
                     orc_factor** out) {
    *out = NULL;
    if (n < 0 || max_steps < 1 || (mode != 0 && mode != 1) || !(drop_tol >= 0.0)) return -1;
    if (rows && mode != 0) return -1;
    for (int32_t s = 1; rows && s < nrows; ++s)
        if (rows[s] <= rows[s - 1]) return -1;
    for (int32_t s = 0; rows && s < nrows; ++s)
        if (rows[s] < 0 || rows[s] >= n) return -1;
    int rc = orc_validate(n, rowptr, col, val);
    if (rc) return rc;
    tables t;
    if ((rc = tables_build(n, rowptr, col, val, &t))) return rc;
    for (int32_t k = 0; k < n; ++k)
        if (t.up0[k] >= 0 && budget[k] < 1) { tables_free(&t); return -1; }

    orc_factor* f = (orc_factor*)calloc(1, sizeof(orc_factor));
    uint64_t* cnt = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1) * 2);
    if (!f || !cnt || !list) { rc = -4; goto fail; }
    f->n = n;
    f->rowptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    f->D = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    f->M = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    f->J = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    f->G = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    f->hops = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    if (!f->rowptr || !f->D || !f->M || !f->J || !f->G || !f->hops) { rc = -4; goto fail; }

    if (mode == 0) {
        int64_t widx = 0;
        int32_t sel = 0;
        for (int32_t k = 0; k < n; ++k) {
            int32_t nlist = 0;
            if (rows) {
                /* only the selected rows are computed; the others stay empty */
                if (sel >= nrows || rows[sel] != k) { f->rowptr[k + 1] = f->nnz; continue; }
                ++sel;
            }
            if (t.up0[k] >= 0) {
                for (uint32_t w = 0; w < budget[k]; ++w) {
                    int32_t end = -1;
                    uint32_t ret = 0;
                    uint64_t h = 0;
                    rc = one_walk(&t, seed, matrix_index, tag, k, w, max_steps, &end, &ret, &h,
                                  NULL, 0, NULL);
                    if (rc) goto fail;
                    if (rec_end && widx < rec_cap) {
                        rec_end[widx] = end;
                        if (rec_ret) rec_ret[widx] = ret;
                        if (rec_len) rec_len[widx] = (uint32_t)h;
                    }
                    ++widx;
                    f->M[k] += 1;
                    f->J[k] += 1 + (uint64_t)ret;
                    f->hops[k] += h;
                    if (end < 0) f->G[k] += 1;
                    else {
                        if (cnt[end] == 0) list[nlist++] = end;
                        cnt[end] += 1;
                    }
                }
            }
            rc = emit_row(f, rowptr, col, val, &t, k, cnt, list, nlist, drop_tol);
            if (rc) goto fail;
            f->rowptr[k + 1] = f->nnz;
        }
    } else {
        /* Walk reuse: all simulated walks first (their extracted sub-walks
         * update other rows' counters), then the factor rows. */
        int64_t path_cap = (int64_t)(max_steps < (1u << 26) ? max_steps : (1u << 26)) + 2;
        int32_t* path = (int32_t*)malloc(sizeof(int32_t) * (size_t)path_cap);
        stacks st = {(int32_t*)malloc(sizeof(int32_t) * (size_t)path_cap),
                     (int64_t*)malloc(sizeof(int64_t) * (size_t)path_cap), path_cap};
        reuse_out o = {f->M, f->J, f->G, NULL, NULL, 0, 0};
        if (!path || !st.node || !st.pos) {
            free(path); free(st.node); free(st.pos);
            rc = -4; goto fail;
        }
        int64_t widx = 0;
        for (int32_t k = 0; k < n && rc == 0; ++k) {
            if (t.up0[k] < 0) continue;
            for (uint32_t w = 0; w < budget[k]; ++w) {
                int32_t end = -1;
                uint32_t ret = 0;
                uint64_t h = 0;
                int64_t plen = 0;
                rc = one_walk(&t, seed, matrix_index, tag, k, w, max_steps, &end, &ret, &h,
                              path, path_cap, &plen);
                if (rc) break;
                if (rec_end && widx < rec_cap) {
                    rec_end[widx] = end;
                    if (rec_ret) rec_ret[widx] = ret;
                    if (rec_len) rec_len[widx] = (uint32_t)h;
                }
                ++widx;
                f->hops[k] += h;
                rc = reuse_walk(path, plen, &st, &o);
                if (rc) break;
            }
        }
        free(path); free(st.node); free(st.pos);
        if (rc) { free(o.hs); free(o.he); goto fail; }
        /* bucket the H updates per start row */
        int64_t* hp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
        int32_t* hend = (int32_t*)malloc(sizeof(int32_t) * (size_t)(o.nh > 0 ? o.nh : 1));
        if (!hp || !hend) { free(hp); free(hend); free(o.hs); free(o.he); rc = -4; goto fail; }
        for (int64_t i = 0; i < o.nh; ++i) hp[o.hs[i] + 1]++;
        for (int32_t k = 0; k < n; ++k) hp[k + 1] += hp[k];
        {
            int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
            if (!fill) { free(hp); free(hend); free(o.hs); free(o.he); rc = -4; goto fail; }
            memcpy(fill, hp, sizeof(int64_t) * (size_t)n);
            for (int64_t i = 0; i < o.nh; ++i) hend[fill[o.hs[i]]++] = o.he[i];
            free(fill);
        }
        free(o.hs); free(o.he);
        for (int32_t k = 0; k < n; ++k) {
            int32_t nlist = 0;
            for (int64_t i = hp[k]; i < hp[k + 1]; ++i) {
                int32_t e = hend[i];
                if (cnt[e] == 0) list[nlist++] = e;
                cnt[e] += 1;
            }
            rc = emit_row(f, rowptr, col, val, &t, k, cnt, list, nlist, drop_tol);
            if (rc) { free(hp); free(hend); goto fail; }
            f->rowptr[k + 1] = f->nnz;
        }
        free(hp); free(hend);
    }
    free(cnt); free(list); tables_free(&t);
    *out = f;
    return 0;
fail:
    free(cnt); free(list); tables_free(&t);
    orc_factor_free(f);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The same build on several host threads.  Rows are independent (Sec. 4: each */
/* row of Y uses only "rows 0..k-1 are homes"), so chunks of consecutive rows  */
/* go to threads in any order; every row runs exactly the walks and the        */
/* emission of the single-thread loop above, and the chunks are concatenated   */
/* in row order afterwards.  The result therefore does not depend on the       */
/* thread count.  Mode 0 only, no per-walk records.                            */
/* ------------------------------------------------------------------------ */
enum { kMtChunkRows = 256 }; /* largest chunk; fewer rows per chunk for short row lists */

typedef struct {
    const tables* t;
    const int32_t *rowptr, *col;
    const double* val;
    const uint32_t* budget;
    uint64_t seed, max_steps;
    uint32_t mi, tag;
    double drop_tol;
    const int32_t* rows;   /* ascending row list (NULL: all rows) */
    int32_t nlist;         /* rows in the list (n when rows == NULL) */
    int64_t nchunks, chunk_rows;
    orc_factor* f;         /* shared per-row arrays D, M, J, G, hops */
    orc_factor* chunk;     /* [nchunks] per-chunk Y entries */
    int64_t* rownnz;       /* [n] entries kept per row */
    atomic_llong next;
    atomic_int err;
} mt_job;

static void* mt_worker(void* arg) {
    mt_job* J = (mt_job*)arg;
    const int32_t n = J->f->n;
    uint64_t* cnt = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1) * 2);
    if (!cnt || !list) {
        atomic_store(&J->err, -4);
        free(cnt); free(list);
        return NULL;
    }
    for (;;) {
        if (atomic_load(&J->err)) break;
        const int64_t c = atomic_fetch_add(&J->next, 1);
        if (c >= J->nchunks) break;
        orc_factor* fc = &J->chunk[c];
        const int64_t s0 = c * J->chunk_rows;
        const int64_t s1 = s0 + J->chunk_rows < J->nlist ? s0 + J->chunk_rows : J->nlist;
        for (int64_t s = s0; s < s1; ++s) {
            const int32_t k = J->rows ? J->rows[s] : (int32_t)s;
            int32_t nlist = 0;
            if (J->t->up0[k] >= 0) {
                for (uint32_t w = 0; w < J->budget[k]; ++w) {
                    int32_t end = -1;
                    uint32_t ret = 0;
                    uint64_t h = 0;
                    int rc = one_walk(J->t, J->seed, J->mi, J->tag, k, w, J->max_steps, &end, &ret,
                                      &h, NULL, 0, NULL);
                    if (rc) { atomic_store(&J->err, rc); goto out; }
                    fc->M[k] += 1;
                    fc->J[k] += 1 + (uint64_t)ret;
                    fc->hops[k] += h;
                    if (end < 0) fc->G[k] += 1;
                    else {
                        if (cnt[end] == 0) list[nlist++] = end;
                        cnt[end] += 1;
                    }
                }
            }
            const int64_t before = fc->nnz;
            int rc = emit_row(fc, J->rowptr, J->col, J->val, J->t, k, cnt, list, nlist, J->drop_tol);
            if (rc) { atomic_store(&J->err, rc); goto out; }
            J->rownnz[k] = fc->nnz - before;
        }
    }
out:
    free(cnt); free(list);
    return NULL;
}

int orc_factor_build_mt(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        const uint32_t* budget, uint64_t seed, uint32_t matrix_index, uint32_t tag,
                        double drop_tol, uint64_t max_steps, const int32_t* rows, int32_t nrows,
                        int32_t nthreads, orc_factor** out) {
    *out = NULL;
    if (n < 0 || max_steps < 1 || !(drop_tol >= 0.0) || nthreads < 1 || nthreads > 1024) return -1;
    for (int32_t s = 1; rows && s < nrows; ++s)
        if (rows[s] <= rows[s - 1]) return -1;
    for (int32_t s = 0; rows && s < nrows; ++s)
        if (rows[s] < 0 || rows[s] >= n) return -1;
    int rc = orc_validate(n, rowptr, col, val);
    if (rc) return rc;
    tables t;
    if ((rc = tables_build(n, rowptr, col, val, &t))) return rc;
    for (int32_t k = 0; k < n; ++k)
        if (t.up0[k] >= 0 && budget[k] < 1) { tables_free(&t); return -1; }
    const size_t nn = (size_t)(n > 0 ? n : 1);
    orc_factor* f = (orc_factor*)calloc(1, sizeof(orc_factor));
    mt_job J;
    memset(&J, 0, sizeof(J));
    pthread_t* th = NULL;
    int started = 0;
    if (!f) { tables_free(&t); return -4; }
    f->n = n;
    f->rowptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    f->D = (double*)calloc(nn, sizeof(double));
    f->M = (uint64_t*)calloc(nn, sizeof(uint64_t));
    f->J = (uint64_t*)calloc(nn, sizeof(uint64_t));
    f->G = (uint64_t*)calloc(nn, sizeof(uint64_t));
    f->hops = (uint64_t*)calloc(nn, sizeof(uint64_t));
    J.nlist = rows ? nrows : n;
    /* about 16 chunks per thread, at most kMtChunkRows rows each */
    J.chunk_rows = (int64_t)J.nlist / ((int64_t)nthreads * 16);
    if (J.chunk_rows < 1) J.chunk_rows = 1;
    if (J.chunk_rows > kMtChunkRows) J.chunk_rows = kMtChunkRows;
    J.nchunks = ((int64_t)J.nlist + J.chunk_rows - 1) / J.chunk_rows;
    J.chunk = (orc_factor*)calloc((size_t)(J.nchunks > 0 ? J.nchunks : 1), sizeof(orc_factor));
    J.rownnz = (int64_t*)calloc(nn, sizeof(int64_t));
    th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!f->rowptr || !f->D || !f->M || !f->J || !f->G || !f->hops || !J.chunk || !J.rownnz || !th) {
        rc = -4;
        goto done;
    }
    for (int64_t c = 0; c < J.nchunks; ++c) {
        J.chunk[c].n = n;
        J.chunk[c].D = f->D; J.chunk[c].M = f->M; J.chunk[c].J = f->J;
        J.chunk[c].G = f->G; J.chunk[c].hops = f->hops;
    }
    J.t = &t; J.rowptr = rowptr; J.col = col; J.val = val; J.budget = budget;
    J.seed = seed; J.max_steps = max_steps; J.mi = matrix_index; J.tag = tag;
    J.drop_tol = drop_tol; J.rows = rows; J.f = f;
    atomic_init(&J.next, 0);
    atomic_init(&J.err, 0);
    for (; started < nthreads; ++started)
        if (pthread_create(&th[started], NULL, mt_worker, &J) != 0) break;
    if (started == 0) mt_worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    if ((rc = atomic_load(&J.err))) goto done;
    /* row pointers, then the chunks' entries in row order */
    for (int32_t k = 0; k < n; ++k) f->rowptr[k + 1] = f->rowptr[k] + J.rownnz[k];
    f->nnz = f->rowptr[n];
    f->cap = f->nnz > 0 ? f->nnz : 1;
    f->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)f->cap);
    f->val = (double*)malloc(sizeof(double) * (size_t)f->cap);
    if (!f->col || !f->val) { rc = -4; goto done; }
    {
        int64_t o = 0;
        for (int64_t c = 0; c < J.nchunks; ++c) {
            if (J.chunk[c].nnz == 0) continue;
            memcpy(f->col + o, J.chunk[c].col, sizeof(int32_t) * (size_t)J.chunk[c].nnz);
            memcpy(f->val + o, J.chunk[c].val, sizeof(double) * (size_t)J.chunk[c].nnz);
            o += J.chunk[c].nnz;
        }
    }
done:
    for (int64_t c = 0; J.chunk && c < J.nchunks; ++c) { free(J.chunk[c].col); free(J.chunk[c].val); }
    free(J.chunk); free(J.rownnz); free(th);
    tables_free(&t);
    if (rc) { orc_factor_free(f); return rc; }
    *out = f;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Preconditioned conjugate gradients (Algorithm 1, "solve"), in the plain     */
/* form of the PCG templates the paper cites for its multiplication count.    */
/* M^-1 r = Y^-1 D^-1 Y^-T r: solve Y^T w = r, v = w / D, solve Y z = v.      */
/* ------------------------------------------------------------------------ */
static void spmv64(int32_t n, const int32_t* rp, const int32_t* ci, const double* a,
                   const double* x, double* y) {
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) s = s + a[p] * x[ci[p]];
        y[i] = s;
    }
}

/* FP32 operator of the mixed mode in excess + difference form: an R-matrix
 * row is A_ii x_i + sum_j A_ij x_j = e_i x_i + sum_{j != i} A_ij (x_j - x_i)
 * with the diagonal excess e_i = A_ii + sum_{j != i} A_ij >= 0 (the ground
 * weight of the walk game, Eq. map).  a[] holds A_ij (j != i) rounded to FP32
 * and, at the diagonal position, e_i computed in FP64 (sum of the row in
 * column order) and rounded to FP32.  Rounding then perturbs each edge weight
 * and each excess by a relative 2^-24 only, so the FP32 operator keeps the
 * near-null space of a weakly grounded matrix; rounding A_ii itself would
 * shift row sums by 2^-24 A_ii, which swamps a small excess. */
static void to_fp32_diff(int32_t n, const int32_t* rp, const int32_t* ci, const double* v,
                         float* a) {
    for (int32_t i = 0; i < n; ++i) {
        double e = 0.0;
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) e = e + v[p];
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) a[p] = ci[p] == i ? (float)e : (float)v[p];
    }
}

static void spmv32(int32_t n, const int32_t* rp, const int32_t* ci, const float* a,
                   const float* x, float* y) {
    for (int32_t i = 0; i < n; ++i) {
        float s = 0.0f;
        const float xi = x[i];
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
            s = s + (ci[p] == i ? a[p] * xi : a[p] * (x[ci[p]] - xi));
        y[i] = s;
    }
}

static void precond64(int32_t n, const int64_t* yrp, const int32_t* yc, const double* yv,
                      const double* D, const double* r, double* w, double* z) {
    /* Y^T w = r by columns of Y^T (rows of Y), last row first */
    for (int32_t i = 0; i < n; ++i) w[i] = r[i];
    for (int32_t k = n - 1; k >= 0; --k)
        for (int64_t p = yrp[k]; p < yrp[k + 1]; ++p) w[yc[p]] = w[yc[p]] - yv[p] * w[k];
    /* Y z = w / D, first row first */
    for (int32_t k = 0; k < n; ++k) {
        double s = w[k] / D[k];
        for (int64_t p = yrp[k]; p < yrp[k + 1]; ++p) s = s - yv[p] * z[yc[p]];
        z[k] = s;
    }
}

static void precond32(int32_t n, const int64_t* yrp, const int32_t* yc, const float* yv,
                      const float* D, const float* r, float* w, float* z) {
    for (int32_t i = 0; i < n; ++i) w[i] = r[i];
    for (int32_t k = n - 1; k >= 0; --k)
        for (int64_t p = yrp[k]; p < yrp[k + 1]; ++p) w[yc[p]] = w[yc[p]] - yv[p] * w[k];
    for (int32_t k = 0; k < n; ++k) {
        float s = w[k] / D[k];
        for (int64_t p = yrp[k]; p < yrp[k + 1]; ++p) s = s - yv[p] * z[yc[p]];
        z[k] = s;
    }
}

static double dot64(int32_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

static double dot32(int32_t n, const float* a, const float* b) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s = s + (double)a[i] * (double)b[i];
    return s;
}

static double true_resid(int32_t n, const int32_t* rp, const int32_t* ci, const double* a,
                         const double* b, const double* x, double* t) {
    spmv64(n, rp, ci, a, x, t);
    for (int32_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
    return sqrt(dot64(n, t, t));
}

static int pcg64(int32_t n, const int32_t* Arp, const int32_t* Acol, const double* Aval,
                 const int64_t* Yrp, const int32_t* Ycol, const double* Yval, const double* D,
                 const double* b, double* x, double tol, int32_t max_iter,
                 int32_t* iters_out, double* relres_out) {
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *r = malloc(sz), *z = malloc(sz), *p = malloc(sz), *q = malloc(sz), *w = malloc(sz);
    if (!r || !z || !p || !q || !w) { free(r); free(z); free(p); free(q); free(w); return -4; }
    int rc = -5;
    for (int32_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double bnorm = sqrt(dot64(n, b, b));
    *iters_out = 0;
    *relres_out = 0.0;
    if (bnorm == 0.0) { rc = 0; goto done; }
    precond64(n, Yrp, Ycol, Yval, D, r, w, z);
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = dot64(n, r, z);
    int32_t it;
    for (it = 1; it <= max_iter; ++it) {
        spmv64(n, Arp, Acol, Aval, p, q);
        double pq = dot64(n, p, q);
        if (!(pq > 0.0)) { rc = -6; break; }
        double alpha = rho / pq;
        for (int32_t i = 0; i < n; ++i) { x[i] = x[i] + alpha * p[i]; r[i] = r[i] - alpha * q[i]; }
        double rn = sqrt(dot64(n, r, r));
        if (rn < tol * bnorm) {
            double tn = true_resid(n, Arp, Acol, Aval, b, x, w);
            if (tn < tol * bnorm) { rc = 0; *iters_out = it; *relres_out = tn / bnorm; goto done; }
        }
        precond64(n, Yrp, Ycol, Yval, D, r, w, z);
        double rho_new = dot64(n, r, z);
        double beta = rho_new / rho;
        rho = rho_new;
        for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    *iters_out = it > max_iter ? max_iter : it;
    *relres_out = true_resid(n, Arp, Acol, Aval, b, x, w) / bnorm;
done:
    free(r); free(z); free(p); free(q); free(w);
    return rc;
}

static int pcg_mixed(int32_t n, const int32_t* Arp, const int32_t* Acol, const double* Aval,
                     const int64_t* Yrp, const int32_t* Ycol, const double* Yval, const double* D,
                     const double* b, double* x, double tol, int32_t max_iter,
                     int32_t refine_every, int32_t* iters_out, double* relres_out) {
    size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t ynnz = Yrp[n], annz = Arp[n];
    float *A32 = malloc(sizeof(float) * (size_t)(annz > 0 ? annz : 1));
    float *Y32 = malloc(sizeof(float) * (size_t)(ynnz > 0 ? ynnz : 1));
    float *D32 = malloc(sizeof(float) * nn);
    float *r = malloc(sizeof(float) * nn), *z = malloc(sizeof(float) * nn);
    float *p = malloc(sizeof(float) * nn), *q = malloc(sizeof(float) * nn);
    float *w = malloc(sizeof(float) * nn);
    double *t = malloc(sizeof(double) * nn);
    int rc = -5;
    if (!A32 || !Y32 || !D32 || !r || !z || !p || !q || !w || !t) { rc = -4; goto done; }
    to_fp32_diff(n, Arp, Acol, Aval, A32);
    for (int64_t i = 0; i < ynnz; ++i) Y32[i] = (float)Yval[i];
    for (int32_t i = 0; i < n; ++i) D32[i] = (float)D[i];
    for (int32_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = (float)b[i]; }
    double bnorm = sqrt(dot64(n, b, b));
    *iters_out = 0;
    *relres_out = 0.0;
    if (bnorm == 0.0) { rc = 0; goto done; }
    precond32(n, Yrp, Ycol, Y32, D32, r, w, z);
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = dot32(n, r, z);
    int32_t it;
    for (it = 1; it <= max_iter; ++it) {
        spmv32(n, Arp, Acol, A32, p, q);
        double pq = dot32(n, p, q);
        if (!(pq > 0.0)) { rc = -6; break; }
        double alpha = rho / pq;
        for (int32_t i = 0; i < n; ++i) {
            x[i] = x[i] + alpha * (double)p[i];
            r[i] = (float)((double)r[i] - alpha * (double)q[i]);
        }
        if (refine_every > 0 && it % refine_every == 0) {
            true_resid(n, Arp, Acol, Aval, b, x, t);
            for (int32_t i = 0; i < n; ++i) r[i] = (float)t[i];
        }
        double rn = sqrt(dot32(n, r, r));
        if (rn < tol * bnorm) {
            double tn = true_resid(n, Arp, Acol, Aval, b, x, t);
            if (tn < tol * bnorm) { rc = 0; *iters_out = it; *relres_out = tn / bnorm; goto done; }
        }
        precond32(n, Yrp, Ycol, Y32, D32, r, w, z);
        double rho_new = dot32(n, r, z);
        double beta = rho_new / rho;
        rho = rho_new;
        for (int32_t i = 0; i < n; ++i) p[i] = (float)((double)z[i] + beta * (double)p[i]);
    }
    *iters_out = it > max_iter ? max_iter : it;
    *relres_out = true_resid(n, Arp, Acol, Aval, b, x, t) / bnorm;
done:
    free(A32); free(Y32); free(D32); free(r); free(z); free(p); free(q); free(w); free(t);
    return rc;
}

int orc_precond_apply(int32_t n, const int64_t* Yrp, const int32_t* Ycol, const double* Yval,
                      const double* D, const double* r, double* z) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!w) return -4;
    precond64(n, Yrp, Ycol, Yval, D, r, w, z);
    free(w);
    return 0;
}

int orc_pcg(int32_t n, const int32_t* Arp, const int32_t* Acol, const double* Aval,
            const int64_t* Yrp, const int32_t* Ycol, const double* Yval, const double* D,
            const double* b, double* x, double tol, int32_t max_iter, int32_t mixed,
            int32_t refine_every, int32_t* iters_out, double* relres_out) {
    if (n < 0 || max_iter < 0 || !(tol >= 0.0)) return -1;
    if (mixed)
        return pcg_mixed(n, Arp, Acol, Aval, Yrp, Ycol, Yval, D, b, x, tol, max_iter,
                         refine_every, iters_out, relres_out);
    return pcg64(n, Arp, Acol, Aval, Yrp, Ycol, Yval, D, b, x, tol, max_iter, iters_out,
                 relres_out);
}


/*
 * Adaptive walk counts of Sec. 5.1 (Eq. lengthdelta): walks from row k run
 * until Delta Xi' sqrt(M) / sigma > z for the mean Xi' and sample standard
 * deviation sigma of their lengths, checked in rounds: min_walks walks first;
 * after each round, if Delta^2 Xi'^2 M > z^2 sigma^2 fails (and M < max_walks),
 * the row's count grows to max(M + 1, ceil(z^2 sigma^2 / (Delta^2 Xi'^2)))
 * (at most max_walks), running walks M, M+1, ...; at most max_rounds rounds.
 * Lengths are the factor walks' hops (walk kind 0).  Sums of lengths and
 * squared lengths are exact integers; the test is FP64 with each operation
 * rounded once.  budget[k] = M_k (0 for rows without an upper neighbour).
 */
int orc_adaptive_budget(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        uint64_t seed, uint32_t matrix_index, double delta, double z,
                        uint32_t min_walks, uint32_t max_walks, int32_t max_rounds,
                        uint64_t max_steps, uint32_t* budget, int32_t* rounds_out) {
    if (n < 0 || !(delta > 0.0) || !(z > 0.0) || min_walks < 2 || max_walks < min_walks ||
        max_walks > 65535u || max_rounds < 1 || max_steps < 1)
        return -1;
    int rc = orc_validate(n, rowptr, col, val);
    if (rc) return rc;
    tables t;
    if ((rc = tables_build(n, rowptr, col, val, &t))) return rc;
    const double d2 = delta * delta, z2 = z * z;
    int32_t rounds_max = 0;
    for (int32_t k = 0; k < n; ++k) {
        budget[k] = 0;
        if (t.up0[k] < 0) continue;
        uint32_t m = 0, inc = min_walks;
        uint64_t s1 = 0, s2 = 0;
        int32_t round;
        for (round = 0; round < max_rounds && inc > 0; ++round) {
            for (uint32_t w = m; w < m + inc; ++w) {
                int32_t end;
                uint32_t ret;
                uint64_t h;
                if ((rc = one_walk(&t, seed, matrix_index, 0, k, w, max_steps, &end, &ret, &h, NULL, 0, NULL))) {
                    tables_free(&t);
                    return rc;
                }
                s1 += h;
                s2 += h * h;
            }
            m += inc;
            inc = 0;
            if (m > 1 && m < max_walks) {
                const double md = (double)m;
                const double mean = (double)s1 / md;
                const double var = ((double)s2 - (double)s1 * mean) / (md - 1.0);
                const double lhs = d2 * (mean * mean) * md;
                const double rhs = z2 * var;
                if (!(lhs > rhs)) {
                    const double need = rhs / (d2 * (mean * mean));
                    uint32_t target = need >= (double)max_walks ? max_walks : (uint32_t)ceil(need);
                    if (target < m + 1) target = m + 1;
                    inc = target - m;
                }
            }
        }
        if (round > rounds_max) rounds_max = round;
        budget[k] = m;
    }
    tables_free(&t);
    if (rounds_out) *rounds_out = rounds_max;
    return 0;
}
