/*
 * FP64 CPU oracle for EpicFlow's sparse-to-dense interpolator
 * (Revaud, Weinzaepfel, Harchaoui, Schmid, "EpicFlow: Edge-Preserving
 * Interpolation of Correspondences for Optical Flow", arXiv:1501.02565).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does.  It shares
 * no code, header or constant with the CUDA path.
 *
 * Every step follows the paper's order (Algorithm 1, LA form of Sec. 3.4):
 *   1. assignment map L and distance D (Sec. 3.4 "Geodesic Voronoi diagram",
 *      distance of Eq. 3) by multi-source Dijkstra on the 8-connected grid;
 *   2. match graph G from neighbouring cells of L (Sec. 3.4 "Approximated
 *      geodesic distance"), edge weight = geodesic distance restricted to
 *      the two cells;
 *   3. N_K(p_m) by Dijkstra on G for every match (Algorithm 1, step 5);
 *   4. weighted affine fit per match (Eq. 2, kernel k_D = exp(-a D) of
 *      Eq. 1), restricted to N_K (Sec. 3.2 "Local interpolation");
 *   5. write-out F(p) = A_{L(p)} p + t_{L(p)} (Algorithm 1 steps 7-8, LA).
 *
 * Readings taken where the paper is silent (each listed in the design notes):
 *   - Eq. 3 is discretised on the 8-connected pixel grid; the step p->q costs
 *     |p-q| * (C(p)+C(q))/2 (trapezoid rule), |p-q| in {1, sqrt 2}.
 *   - pixel centres are integer coordinates, x = column, y = row; a match's
 *     source pixel is (floor(x+0.5), floor(y+0.5)).
 *   - "neighbours in L" means 8-adjacent pixels with different labels.
 *   - ties go to the smallest match index everywhere (labels, K-th neighbour).
 *   - N_K(p_m) contains p_m itself (graph distance 0).
 *   - Eq. 2 is solved as a weighted least-squares problem whose rows are
 *     scaled by k, i.e. it minimises sum k^2 |A p + t - p'|^2
 *     (weight_squared = 1); weight_squared = 0 minimises sum k |.|^2.
 *   - Eq. 1 averages the matches' correspondences expressed as flows,
 *     u_n = p'_n - p_n, so the estimate at p_m is a flow; the per-cell
 *     property of Sec. 3.4 then makes the NW flow constant over a cell.
 *     (Averaging the positions p'_n literally would shift every estimate
 *     by the kernel-weighted centroid offset of the neighbours, a bias of
 *     several pixels that the NW accuracy the paper reports rules out.)
 *   - a fit with fewer than 3 neighbours or det(M) <= 1e-10 (tr M / 3)^3
 *     falls back to that Nadaraya-Watson flow at p_m, held constant over
 *     the cell.
 *   - a match whose source pixel is owned by a smaller-index duplicate has an
 *     empty cell; it is joined to the owner by an edge of weight D = 0.
 *
 * Model layout (per match m, 6 doubles): c_u, c_v, b11, b12, b21, b22 with
 *   flow(p) = F(p) - p = c + B (p - p_m).
 * Fitting the flow u = p' - p with an affine function of p is the same
 * least-squares problem as fitting p' (the residuals are identical with
 * A = I + B), and centring on p_m only re-parametrises t.
 *
 * Compiled with -ffp-contract=off so that x86-64 and aarch64 hosts produce
 * identical results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID -1
#define ORACLE_ERR_CAPACITY -2
#define ORACLE_ERR_NOMEM -3

/* ------------------------------------------------------------------------ */
/* binary min-heap on the lexicographic key (d, tag), payload node           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double d;
    int tag;
    int node;
} hitem;

typedef struct {
    hitem *a;
    long n, cap;
} heap;

static int key_less(const hitem *x, const hitem *y) {
    if (x->d < y->d) return 1;
    if (x->d > y->d) return 0;
    return x->tag < y->tag;
}

static int heap_push(heap *h, double d, int tag, int node) {
    if (h->n == h->cap) {
        long nc = h->cap ? 2 * h->cap : 1024;
        hitem *na = (hitem *)realloc(h->a, (size_t)nc * sizeof(hitem));
        if (!na) return ORACLE_ERR_NOMEM;
        h->a = na;
        h->cap = nc;
    }
    long i = h->n++;
    hitem it = {d, tag, node};
    while (i > 0) {
        long p = (i - 1) / 2;
        if (!key_less(&it, &h->a[p])) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = it;
    return ORACLE_OK;
}

static hitem heap_pop(heap *h) {
    hitem top = h->a[0];
    hitem last = h->a[--h->n];
    long i = 0;
    for (;;) {
        long l = 2 * i + 1, r = l + 1, s = i;
        const hitem *best = &last;
        if (l < h->n && key_less(&h->a[l], best)) { s = l; best = &h->a[l]; }
        if (r < h->n && key_less(&h->a[r], best)) { s = r; }
        if (s == i) break;
        h->a[i] = h->a[s];
        i = s;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3 on the 8-connected grid                                             */
/* ------------------------------------------------------------------------ */

static const int NB_DX[8] = {1, -1, 0, 0, 1, 1, -1, -1};
static const int NB_DY[8] = {0, 0, 1, -1, 1, -1, 1, -1};

/* cost of the grid step between neighbouring pixels p and q (trapezoid rule
 * on the segment joining their centres) */
static double step_cost(const float *C, long p, long q, int diagonal) {
    double len = diagonal ? sqrt(2.0) : 1.0;
    return len * ((double)C[p] + (double)C[q]) * 0.5;
}

static int seed_pixel(const float *matches, int m, int H, int W, long *pix) {
    double x = floor((double)matches[4 * m + 0] + 0.5);
    double y = floor((double)matches[4 * m + 1] + 0.5);
    if (!(x >= 0 && x < W && y >= 0 && y < H)) return ORACLE_ERR_INVALID;
    *pix = (long)y * W + (long)x;
    return ORACLE_OK;
}

/*
 * Geodesic Voronoi assignment (Sec. 3.4): for every pixel p,
 *   L(p) = argmin_m D_G(p, p_m)   and   D(p) = min_m D_G(p, p_m),
 * ties to the smallest m.  Multi-source Dijkstra whose heap key is the pair
 * (distance, match index), compared lexicographically.
 */
int epic_oracle_geodesic(const float *C, int H, int W, const float *matches,
                         int N, double *D, int *L) {
    if (H < 1 || W < 1 || N < 1) return ORACLE_ERR_INVALID;
    long P = (long)H * W;
    for (long p = 0; p < P; ++p) {
        if (!(C[p] >= 0.0f) || isinf(C[p])) return ORACLE_ERR_INVALID;
        D[p] = INFINITY;
        L[p] = -1;
    }
    char *done = (char *)calloc((size_t)P, 1);
    if (!done) return ORACLE_ERR_NOMEM;
    heap h = {0};
    int rc = ORACLE_OK;
    for (int m = 0; m < N && rc == ORACLE_OK; ++m) {
        long pix;
        rc = seed_pixel(matches, m, H, W, &pix);
        if (rc == ORACLE_OK) rc = heap_push(&h, 0.0, m, (int)pix);
    }
    while (rc == ORACLE_OK && h.n > 0) {
        hitem it = heap_pop(&h);
        long p = it.node;
        if (done[p]) continue;
        done[p] = 1;
        D[p] = it.d;
        L[p] = it.tag;
        int x = (int)(p % W), y = (int)(p / W);
        for (int k = 0; k < 8; ++k) {
            int qx = x + NB_DX[k], qy = y + NB_DY[k];
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
            long q = (long)qy * W + qx;
            if (done[q]) continue;
            double nd = it.d + step_cost(C, p, q, k >= 4);
            if (nd < D[q] || (nd == D[q] && it.tag < L[q])) {
                D[q] = nd;
                L[q] = it.tag;
                rc = heap_push(&h, nd, it.tag, (int)q);
                if (rc != ORACLE_OK) break;
            }
        }
    }
    free(h.a);
    free(done);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* match graph G (Sec. 3.4)                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t key; /* m * N + n, m < n */
    double w;
} cand;

static int cand_cmp(const void *a, const void *b) {
    const cand *x = (const cand *)a, *y = (const cand *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return 0;
}

/*
 * Nodes are the matches; m and n are joined when their cells touch (some
 * 8-adjacent pixels p, q with L(p) = m, L(q) = n).  The weight is the
 * geodesic distance from p_m to p_n with the path restricted to the two
 * cells, which equals the minimum over touching pairs of
 * D(p) + step(p, q) + D(q): a shortest path from a seed to a pixel of its
 * own cell stays inside that cell, and any path inside the union crosses
 * from one cell to the other at some touching pair.
 *
 * Output: edges sorted by (m, n) with m < n.  Returns the edge count, or
 * ORACLE_ERR_CAPACITY if more than cap edges would be written.
 */
long epic_oracle_graph(const float *C, int H, int W, const double *D,
                       const int *L, const float *matches, int N, int *em,
                       int *en, double *ew, long cap) {
    long P = (long)H * W;
    long ncand_cap = 4 * P + N;
    cand *cs = (cand *)malloc((size_t)ncand_cap * sizeof(cand));
    if (!cs) return ORACLE_ERR_NOMEM;
    long nc = 0;
    /* the four forward neighbours cover each unordered pixel pair once */
    static const int FDX[4] = {1, -1, 0, 1};
    static const int FDY[4] = {0, 1, 1, 1};
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            for (int k = 0; k < 4; ++k) {
                int qx = x + FDX[k], qy = y + FDY[k];
                if (qx < 0 || qx >= W || qy >= H) continue;
                long q = (long)qy * W + qx;
                if (L[p] == L[q]) continue;
                int m = L[p] < L[q] ? L[p] : L[q];
                int n = L[p] < L[q] ? L[q] : L[p];
                cs[nc].key = (int64_t)m * N + n;
                cs[nc].w = D[p] + step_cost(C, p, q, FDX[k] != 0 && FDY[k] != 0) + D[q];
                ++nc;
            }
        }
    }
    /* a duplicate source pixel leaves the larger-index match with an empty
     * cell; join it to the pixel's owner at distance D = 0 */
    for (int m = 0; m < N; ++m) {
        long pix;
        if (seed_pixel(matches, m, H, W, &pix) != ORACLE_OK) {
            free(cs);
            return ORACLE_ERR_INVALID;
        }
        if (L[pix] != m) {
            int a = L[pix] < m ? L[pix] : m;
            int b = L[pix] < m ? m : L[pix];
            cs[nc].key = (int64_t)a * N + b;
            cs[nc].w = D[pix];
            ++nc;
        }
    }
    qsort(cs, (size_t)nc, sizeof(cand), cand_cmp);
    long ne = 0;
    for (long i = 0; i < nc; ++i) {
        if (i > 0 && cs[i].key == cs[i - 1].key) continue; /* sorted: first is min */
        if (ne >= cap) {
            free(cs);
            return ORACLE_ERR_CAPACITY;
        }
        em[ne] = (int)(cs[i].key / N);
        en[ne] = (int)(cs[i].key % N);
        ew[ne] = cs[i].w;
        ++ne;
    }
    free(cs);
    return ne;
}

/* ------------------------------------------------------------------------ */
/* N_K(p_m): Dijkstra on G from every match (Algorithm 1, step 5)            */
/* ------------------------------------------------------------------------ */

/*
 * idx[m*K + j], dist[m*K + j] for j < count[m]: the matches in the order
 * Dijkstra settles them from m, key (graph distance, match index).  The first
 * entry is m itself at distance 0.  count[m] = min(K, size of m's component).
 */
int epic_oracle_knn(int N, long E, const int *em, const int *en,
                    const double *ew, int K, int *idx, double *dist,
                    int *count) {
    if (N < 1 || K < 1) return ORACLE_ERR_INVALID;
    long *rp = (long *)calloc((size_t)N + 1, sizeof(long));
    int *col = (int *)malloc((size_t)(2 * E + 1) * sizeof(int));
    double *wt = (double *)malloc((size_t)(2 * E + 1) * sizeof(double));
    double *best = (double *)malloc((size_t)N * sizeof(double));
    int *seen = (int *)malloc((size_t)N * sizeof(int));
    long *fill = (long *)malloc((size_t)N * sizeof(long));
    int rc = ORACLE_OK;
    if (!rp || !col || !wt || !best || !seen || !fill) {
        rc = ORACLE_ERR_NOMEM;
        goto out;
    }
    for (long e = 0; e < E; ++e) {
        rp[em[e] + 1]++;
        rp[en[e] + 1]++;
    }
    for (int i = 0; i < N; ++i) rp[i + 1] += rp[i];
    for (int i = 0; i < N; ++i) fill[i] = rp[i];
    for (long e = 0; e < E; ++e) {
        col[fill[em[e]]] = en[e];
        wt[fill[em[e]]++] = ew[e];
        col[fill[en[e]]] = em[e];
        wt[fill[en[e]]++] = ew[e];
    }
    for (int i = 0; i < N; ++i) seen[i] = -1;
    heap h = {0};
    for (int m = 0; m < N && rc == ORACLE_OK; ++m) {
        /* seen[v] == m marks v as touched in this search; best[v] holds its
         * tentative distance, -1 in seen-after-settling is tracked by sign */
        h.n = 0;
        int c = 0;
        rc = heap_push(&h, 0.0, m, m);
        seen[m] = m;
        best[m] = 0.0;
        while (rc == ORACLE_OK && h.n > 0 && c < K) {
            hitem it = heap_pop(&h);
            int v = it.node;
            if (it.d > best[v]) continue;          /* stale entry */
            if (best[v] < 0) continue;             /* settled already */
            idx[(long)m * K + c] = v;
            dist[(long)m * K + c] = it.d;
            ++c;
            best[v] = -1.0 - it.d;                 /* mark settled */
            for (long j = rp[v]; j < rp[v + 1]; ++j) {
                int u = col[j];
                double nd = it.d + wt[j];
                if (seen[u] == m) {
                    if (best[u] < 0) continue;     /* settled */
                    if (!(nd < best[u])) continue;
                } else {
                    seen[u] = m;
                }
                best[u] = nd;
                rc = heap_push(&h, nd, u, u);
                if (rc != ORACLE_OK) break;
            }
        }
        count[m] = c;
    }
    free(h.a);
out:
    free(rp);
    free(col);
    free(wt);
    free(best);
    free(seen);
    free(fill);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* per-match locally-weighted affine fit (Eq. 2 restricted to N_K)           */
/* ------------------------------------------------------------------------ */

static double det3(const double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* Gaussian elimination with partial pivoting on [M | r1 r2] (textbook). */
static void solve3x2(const double Min[3][3], const double r1[3],
                     const double r2[3], double x1[3], double x2[3]) {
    double A[3][5];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) A[i][j] = Min[i][j];
        A[i][3] = r1[i];
        A[i][4] = r2[i];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 5; ++j) {
                double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        for (int r = c + 1; r < 3; ++r) {
            double f = A[r][c] / A[c][c];
            for (int j = c; j < 5; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = 2; i >= 0; --i) {
        double s1 = A[i][3], s2 = A[i][4];
        for (int j = i + 1; j < 3; ++j) {
            s1 -= A[i][j] * x1[j];
            s2 -= A[i][j] * x2[j];
        }
        x1[i] = s1 / A[i][i];
        x2[i] = s2 / A[i][i];
    }
}

/*
 * Locally-weighted affine fit centred at (xc, yc) over c neighbours n (rows
 * of `matches`) at distances d_n:
 *   k_n = exp(-a d_n)                       (kernel of Eq. 1)
 *   w_n = k_n^2  (weight_squared = 1)  or  k_n  (weight_squared = 0)
 *   minimise sum_n w_n | B (p_n - p_c) + c - (p'_n - p_n) |^2   (Eq. 2)
 * through the 3x3 normal equations in (x~, y~, 1), x~ = x_n - xc.
 * *fallback = 1 when the fit is degenerate and the Nadaraya-Watson estimate
 * (Eq. 1) is used instead: c = sum k u_n / sum k with u_n = p'_n - p_n
 * (Eq. 1's kernel k, not squared), B = 0.  *detratio = det M / (tr M / 3)^3
 * (0 when fewer than 3 neighbours).
 */
static void fit_at(double xc, double yc, const float *matches, int c,
                   const int *nbr, const double *dist, double a,
                   int weight_squared, double *out, int *fallback,
                   double *detratio) {
    double M[3][3] = {{0}}, ru[3] = {0}, rv[3] = {0};
    double sw = 0, swu = 0, swv = 0;
    for (int j = 0; j < c; ++j) {
        int n = nbr[j];
        double k = exp(-a * dist[j]);
        double w = weight_squared ? k * k : k;
        double xn = matches[4 * n + 0], yn = matches[4 * n + 1];
        double u = (double)matches[4 * n + 2] - xn;
        double v = (double)matches[4 * n + 3] - yn;
        double phi[3] = {xn - xc, yn - yc, 1.0};
        for (int r = 0; r < 3; ++r) {
            for (int s = 0; s < 3; ++s) M[r][s] += w * phi[r] * phi[s];
            ru[r] += w * phi[r] * u;
            rv[r] += w * phi[r] * v;
        }
        sw += k;
        swu += k * u;
        swv += k * v;
    }
    double tr = M[0][0] + M[1][1] + M[2][2];
    double det = det3(M);
    double scale = (tr / 3.0) * (tr / 3.0) * (tr / 3.0);
    *detratio = (c >= 3 && scale > 0) ? det / scale : 0.0;
    if (c < 3 || !(det > 1e-10 * scale)) {
        *fallback = 1;
        out[0] = swu / sw;
        out[1] = swv / sw;
        out[2] = out[3] = out[4] = out[5] = 0.0;
    } else {
        double bu[3], bv[3];
        solve3x2(M, ru, rv, bu, bv);
        *fallback = 0;
        out[0] = bu[2];
        out[1] = bv[2];
        out[2] = bu[0];
        out[3] = bu[1];
        out[4] = bv[0];
        out[5] = bv[1];
    }
}

/* Per-match fit (Sec. 3.4): centre p_m, neighbours N_K(p_m) on G. */
int epic_oracle_fit(int N, const float *matches, int K, const int *idx,
                    const double *dist, const int *count, double a,
                    int weight_squared, double *model, int *fallback,
                    double *detratio) {
    if (N < 1 || K < 1 || !(a > 0)) return ORACLE_ERR_INVALID;
    for (int m = 0; m < N; ++m)
        fit_at(matches[4 * m + 0], matches[4 * m + 1], matches, count[m],
               idx + (long)m * K, dist + (long)m * K, a, weight_squared,
               model + 6L * m, fallback + m, detratio + m);
    return ORACLE_OK;
}

/* Per-point fit (the exact variant of Sec. 5.2, estimation per pixel):
 * centre (centres[2i], centres[2i+1]), neighbours idx/dist row i. */
int epic_oracle_fit_points(int Np, const double *centres, int N,
                           const float *matches, int K, const int *idx,
                           const double *dist, const int *count, double a,
                           int weight_squared, double *model, int *fallback,
                           double *detratio) {
    if (Np < 0 || N < 1 || K < 1 || !(a > 0)) return ORACLE_ERR_INVALID;
    for (long i = 0; i < Np; ++i) {
        for (int j = 0; j < count[i]; ++j)
            if (idx[i * K + j] < 0 || idx[i * K + j] >= N) return ORACLE_ERR_INVALID;
        fit_at(centres[2 * i], centres[2 * i + 1], matches, count[i], idx + i * K,
               dist + i * K, a, weight_squared, model + 6 * i, fallback + i,
               detratio + i);
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* dense write-out (Algorithm 1, steps 7-8, LA form)                          */
/* ------------------------------------------------------------------------ */

/* flow[(y*W + x)*2 + {0,1}] = c_m + B_m ((x, y) - p_m),  m = L(x, y). */
int epic_oracle_writeout(int H, int W, const int *L, int N,
                         const float *matches, const double *model,
                         double *flow) {
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            int m = L[p];
            if (m < 0 || m >= N) return ORACLE_ERR_INVALID;
            const double *md = model + 6L * m;
            double dx = x - (double)matches[4 * m + 0];
            double dy = y - (double)matches[4 * m + 1];
            flow[2 * p + 0] = md[0] + md[2] * dx + md[3] * dy;
            flow[2 * p + 1] = md[1] + md[4] * dx + md[5] * dy;
        }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Nadaraya-Watson estimate at every match (Eq. 1 restricted to N_K)         */
/* ------------------------------------------------------------------------ */

/* nw[2m], nw[2m+1] = sum_n k_n u_n / sum_n k_n with k_n = exp(-a d_n) and
 * u_n = p'_n - p_n the flow of neighbour n. */
int epic_oracle_nw(int N, const float *matches, int K, const int *idx,
                   const double *dist, const int *count, double a,
                   double *nw) {
    if (N < 1 || K < 1 || !(a > 0)) return ORACLE_ERR_INVALID;
    for (int m = 0; m < N; ++m) {
        double s = 0, sx = 0, sy = 0;
        for (int j = 0; j < count[m]; ++j) {
            int n = idx[(long)m * K + j];
            double k = exp(-a * dist[(long)m * K + j]);
            s += k;
            sx += k * ((double)matches[4 * n + 2] - (double)matches[4 * n + 0]);
            sy += k * ((double)matches[4 * n + 3] - (double)matches[4 * n + 1]);
        }
        nw[2 * m + 0] = sx / s;
        nw[2 * m + 1] = sy / s;
    }
    return ORACLE_OK;
}
