/*
 * Oracle for the Laplace-Beltrami double-layer Nystrom system on the sphere
 * (Kropinski & Nigam, "Fast integral equation methods for the Laplace-Beltrami
 * equation on the sphere").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code with
 * the CUDA path and is deliberately plain: every entry of the bordered matrix
 * is computed from its definition in the 3D sphere form, sums run in index
 * order, in IEEE double precision, compiled without contraction of a*b+c.
 *
 * Conventions (the paper's printed signs and indices are garbled in places;
 * these readings are pinned by the tests):
 *   - nodes x_j on island k are equispaced in the curve parameter alpha,
 *     h_k = 2 pi / N_k, and the curve runs counter-clockwise about the
 *     island centre seen from outside the sphere, so n' ds' = x_j x x'_j d alpha
 *     points into the island (out of the domain, Fig. 1 / Sec. 2).
 *   - double-layer kernel (Sec. 2, Eq. kern1): (1/2pi) d/dn' log|x - x'| ds'
 *       = -(1/2pi) (x - x')·(x' x x'_alpha) / |x - x'|^2 d alpha.
 *   - its diagonal limit (Appendix A, by l'Hopital twice, with the normal above):
 *       -(1/4pi) x·(x' x x'') / |x'|^2 d alpha.
 *   - Nystrom system in the paper's doubled form (Sec. 5, Eq. disc_sphere and
 *     matrix_eqns): rows i < N:  sigma_i + 2 sum_j K_ij sigma_j
 *                                + 2 sum_m G(x_i, c_m) a_m = 2 g_i,
 *     rows N + r (r = 0..M-2): sum of sigma over island r+1 = 0 (Eq. disc_constr,
 *     unweighted, the first island exempt); row N+M-1: sum_m a_m = 0 (Eq. sum_ak).
 *   - G(x, y) = -(1/2pi) log|x - y| + (1/4pi) log 2 (Sec. 1.1, Eq. greens_func).
 *   - evaluation off the curves (Eq. u_multi): u(t) = sum_j K(t, x_j) sigma_j
 *     + sum_m a_m G(t, c_m), with no jump term.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ---- small vector helpers ---------------------------------------------- */
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Generalized fundamental solution, Sec. 1.1 Eq. (greens_func). */
double orc_green(const double *x, const double *y)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r = sqrt(dot3(d, d));
    return -log(r) / (2.0 * ORC_PI) + log(2.0) / (4.0 * ORC_PI);
}

/* Double-layer kernel per unit alpha at target t from node (xj, dxj):
 * -(1/2pi) (t - xj)·(xj x dxj) / |t - xj|^2   (Sec. 2, Eq. kern1). */
static double dl_kernel(const double *t, const double *xj, const double *dxj)
{
    double n[3], d[3];
    cross3(xj, dxj, n);
    d[0] = t[0] - xj[0];
    d[1] = t[1] - xj[1];
    d[2] = t[2] - xj[2];
    return -dot3(d, n) / (2.0 * ORC_PI * dot3(d, d));
}

/* Diagonal limit per unit alpha (Appendix A): -(1/4pi) x·(x' x x'')/|x'|^2. */
static double dl_diag(const double *x, const double *dx, const double *d2x)
{
    double c[3];
    cross3(dx, d2x, c);
    return -dot3(x, c) / (4.0 * ORC_PI * dot3(dx, dx));
}

static int island_of(int M, const int64_t *ptr, int64_t j)
{
    int lo = 0, hi = M - 1;
    while (lo < hi) { /* largest k with ptr[k] <= j */
        int mid = (lo + hi + 1) / 2;
        if (ptr[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* One entry of the bordered matrix (Sec. 5, Eq. matrix_eqns), row i, column j. */
double orc_entry(int64_t N, int M, const int64_t *ptr, const double *x, const double *dx,
                 const double *d2x, const double *c, int64_t i, int64_t j)
{
    if (i < N) {
        if (j < N) {
            int kj = island_of(M, ptr, j);
            double h = 2.0 * ORC_PI / (double)(ptr[kj + 1] - ptr[kj]);
            if (i == j)
                return 1.0 + 2.0 * h * dl_diag(&x[3 * i], &dx[3 * i], &d2x[3 * i]);
            return 2.0 * h * dl_kernel(&x[3 * i], &x[3 * j], &dx[3 * j]);
        }
        return 2.0 * orc_green(&x[3 * i], &c[3 * (j - N)]);
    }
    int64_t r = i - N;
    if (r < M - 1) {
        if (j >= N) return 0.0;
        return (island_of(M, ptr, j) == r + 1) ? 1.0 : 0.0;
    }
    return (j >= N) ? 1.0 : 0.0;
}

/* Dense (N+M) x (N+M) row-major bordered matrix. */
void orc_matrix(int64_t N, int M, const int64_t *ptr, const double *x, const double *dx,
                const double *d2x, const double *c, double *A)
{
    int64_t n = N + M;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            A[i * n + j] = orc_entry(N, M, ptr, x, dx, d2x, c, i, j);
}

/* Rows `rows[0..nrows)` of the matvec, entries computed on the fly.
 * op 0: bordered matrix times v (v has N+M entries);
 * op 1: the density block only, (I + 2K) v (v has N entries; rows must be < N). */
void orc_apply_rows(int64_t N, int M, const int64_t *ptr, const double *x, const double *dx,
                    const double *d2x, const double *c, int op, const double *v,
                    int64_t nrows, const int64_t *rows, double *out)
{
    int64_t ncol = (op == 0) ? N + M : N;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nrows; q++) {
        int64_t i = rows[q];
        double s = 0.0;
        for (int64_t j = 0; j < ncol; j++)
            s += orc_entry(N, M, ptr, x, dx, d2x, c, i, j) * v[j];
        out[q] = s;
    }
}

/* u at off-curve targets (Eq. u_multi): sum_j h_j K(t, x_j) sigma_j + sum_m a_m G(t, c_m). */
void orc_evaluate(int64_t N, int M, const int64_t *ptr, const double *x, const double *dx,
                  const double *c, const double *sigma, const double *a, int64_t T,
                  const double *t, double *u)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < T; q++) {
        double s = 0.0;
        for (int k = 0; k < M; k++) {
            double h = 2.0 * ORC_PI / (double)(ptr[k + 1] - ptr[k]);
            for (int64_t j = ptr[k]; j < ptr[k + 1]; j++)
                s += h * dl_kernel(&t[3 * q], &x[3 * j], &dx[3 * j]) * sigma[j];
        }
        for (int m = 0; m < M; m++)
            s += a[m] * orc_green(&t[3 * q], &c[3 * m]);
        u[q] = s;
    }
}

/* sum_s gamma_s G(t_q, p_s) at T points. */
void orc_green_sum(int64_t T, const double *t, int64_t S, const double *p, const double *gamma,
                   double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < T; q++) {
        double s = 0.0;
        for (int64_t k = 0; k < S; k++)
            s += gamma[k] * orc_green(&t[3 * q], &p[3 * k]);
        out[q] = s;
    }
}

/* ---- stereographic projection (Sec. 3) --------------------------------- */
/* xi = (x1 + i x2) / (1 - x3): written as two correctly rounded divisions by w = 1 - x3. */
void orc_project(int64_t N, const double *x, double *xi /* N x 2 */)
{
    for (int64_t j = 0; j < N; j++) {
        double w = 1.0 - x[3 * j + 2];
        xi[2 * j] = x[3 * j] / w;
        xi[2 * j + 1] = x[3 * j + 1] / w;
    }
}

/* ---- reference quadtree -------------------------------------------------
 * Integer specification (shared by the CUDA build, written independently):
 *   L = max(xmax - xmin, ymax - ymin) * (1 + 2^-20)   (L = 1 if that is 0)
 *   cell = min(2^D - 1, floor((v - vmin) / L * 2^D))  in IEEE double
 *   key  = bit-interleave, y bit above x bit at every level
 *   nodes sorted by (key, original index)
 *   a box at level l is split while it holds more than `leaf` nodes and l < D;
 *   empty children are dropped; boxes are numbered level by level, within a
 *   level in Morton order.                                                   */
typedef struct {
    uint64_t key;
    int64_t idx;
} kv_t;

static int cmp_kv(const void *a, const void *b)
{
    const kv_t *p = (const kv_t *)a, *q = (const kv_t *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

static uint64_t interleave(uint64_t cx, uint64_t cy, int D)
{
    uint64_t k = 0;
    for (int b = 0; b < D; b++) {
        k |= ((cx >> b) & 1ull) << (2 * b);
        k |= ((cy >> b) & 1ull) << (2 * b + 1);
    }
    return k;
}

/* Returns the number of boxes, or -1 if more than `cap` would be needed.
 * bbox_out = {xmin, ymin, L}. */
int64_t orc_tree(int64_t N, const double *xi, int leaf, int D, int64_t cap,
                 int64_t *perm, uint64_t *keys_sorted, double *bbox_out,
                 int32_t *level, int64_t *ix, int64_t *iy, int64_t *parent,
                 int64_t *first_child, int32_t *nchild, int64_t *begin, int64_t *end)
{
    double xmin = xi[0], xmax = xi[0], ymin = xi[1], ymax = xi[1];
    for (int64_t j = 1; j < N; j++) {
        if (xi[2 * j] < xmin) xmin = xi[2 * j];
        if (xi[2 * j] > xmax) xmax = xi[2 * j];
        if (xi[2 * j + 1] < ymin) ymin = xi[2 * j + 1];
        if (xi[2 * j + 1] > ymax) ymax = xi[2 * j + 1];
    }
    double L = (xmax - xmin > ymax - ymin) ? xmax - xmin : ymax - ymin;
    L = L * (1.0 + ldexp(1.0, -20));
    if (!(L > 0.0)) L = 1.0;
    bbox_out[0] = xmin;
    bbox_out[1] = ymin;
    bbox_out[2] = L;
    double scale = ldexp(1.0, D);
    uint64_t cmax = (1ull << D) - 1ull;
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t j = 0; j < N; j++) {
        double fx = floor((xi[2 * j] - xmin) / L * scale);
        double fy = floor((xi[2 * j + 1] - ymin) / L * scale);
        uint64_t cx = (uint64_t)fx, cy = (uint64_t)fy;
        if (cx > cmax) cx = cmax;
        if (cy > cmax) cy = cmax;
        kv[j].key = interleave(cx, cy, D);
        kv[j].idx = j;
    }
    qsort(kv, (size_t)N, sizeof(kv_t), cmp_kv);
    for (int64_t j = 0; j < N; j++) {
        perm[j] = kv[j].idx;
        keys_sorted[j] = kv[j].key;
    }
    free(kv);

    int64_t nb = 1;
    if (cap < 1) return -1;
    level[0] = 0; ix[0] = 0; iy[0] = 0; parent[0] = -1;
    first_child[0] = -1; nchild[0] = 0; begin[0] = 0; end[0] = N;
    for (int64_t b = 0; b < nb; b++) {
        int l = level[b];
        if (end[b] - begin[b] <= leaf || l >= D) continue;
        int shift = 2 * (D - l - 1);
        int64_t s = begin[b];
        for (int d = 0; d < 4; d++) {
            int64_t e = s;
            while (e < end[b] && (int)((keys_sorted[e] >> shift) & 3ull) == d) e++;
            if (e > s) {
                if (nb >= cap) return -1;
                if (nchild[b] == 0) first_child[b] = nb;
                nchild[b]++;
                level[nb] = l + 1;
                ix[nb] = 2 * ix[b] + (d & 1);
                iy[nb] = 2 * iy[b] + (d >> 1);
                parent[nb] = b;
                first_child[nb] = -1;
                nchild[nb] = 0;
                begin[nb] = s;
                end[nb] = e;
                nb++;
            }
            s = e;
        }
    }
    return nb;
}

/* Closed boxes touch or overlap (integer test at the finer level). */
static int boxes_touch(int la, int64_t xa, int64_t ya, int lb, int64_t xb, int64_t yb)
{
    if (la > lb) {
        int t = la; la = lb; lb = t;
        int64_t u = xa; xa = xb; xb = u;
        u = ya; ya = yb; yb = u;
    }
    int s = lb - la;
    int64_t lo_x = xa << s, hi_x = (xa + 1) << s;
    int64_t lo_y = ya << s, hi_y = (ya + 1) << s;
    return (xb <= hi_x) && (xb + 1 >= lo_x) && (yb <= hi_y) && (yb + 1 >= lo_y);
}

/* Interaction lists by brute force over all box pairs (adaptive FMM,
 * Carrier-Greengard-Rokhlin), O(B^2):
 *   U(b), b leaf:   leaves touching b, b included;
 *   V(b):           same-level boxes not touching b whose parents touch (or equal) b's parent;
 *   W(b), b leaf:   boxes d deeper than b, not touching b, whose parent touches b;
 *   X(b):           leaves x shallower than b, not touching b, touching b's parent.
 * kind 0..3 = U, V, W, X.  Output in CSR form, entries ascending.  Returns the
 * total count, or -1 if it exceeds cap.  ptr_out has nb+1 entries. */
int64_t orc_lists(int64_t nb, const int32_t *level, const int64_t *ix, const int64_t *iy,
                  const int64_t *parent, const int32_t *nchild, int kind, int64_t cap,
                  int64_t *ptr_out, int64_t *idx_out)
{
    int64_t cnt = 0;
    for (int64_t b = 0; b < nb; b++) {
        ptr_out[b] = cnt;
        int is_leaf_b = nchild[b] == 0;
        if ((kind == 0 || kind == 2) && !is_leaf_b) continue;
        for (int64_t o = 0; o < nb; o++) {
            int take = 0;
            if (kind == 0) {
                take = nchild[o] == 0 && boxes_touch(level[b], ix[b], iy[b], level[o], ix[o], iy[o]);
            } else if (kind == 1) {
                if (level[o] == level[b] && level[b] > 0 && o != b) {
                    int64_t pb = parent[b], po = parent[o];
                    take = !boxes_touch(level[b], ix[b], iy[b], level[o], ix[o], iy[o]) &&
                           boxes_touch(level[pb], ix[pb], iy[pb], level[po], ix[po], iy[po]);
                }
            } else if (kind == 2) {
                if (level[o] > level[b]) {
                    int64_t po = parent[o];
                    take = !boxes_touch(level[b], ix[b], iy[b], level[o], ix[o], iy[o]) &&
                           boxes_touch(level[b], ix[b], iy[b], level[po], ix[po], iy[po]);
                }
            } else {
                if (nchild[o] == 0 && level[o] < level[b]) {
                    int64_t pb = parent[b];
                    take = !boxes_touch(level[b], ix[b], iy[b], level[o], ix[o], iy[o]) &&
                           boxes_touch(level[pb], ix[pb], iy[pb], level[o], ix[o], iy[o]);
                }
            }
            if (take) {
                if (cnt >= cap) return -1;
                idx_out[cnt++] = o;
            }
        }
    }
    ptr_out[nb] = cnt;
    return cnt;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
