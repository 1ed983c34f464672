/*
 * CPU oracle for the nearest-points search and per-point covariance step of
 * GICP-style scan registration (Sec. III-C1 "Efficient registration method",
 * Eq. 18-20; the step moved to the GPU in Sec. III-C1 and Sec. IV-E1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain definition that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never does,
 * and the two share no source, header, table or helper.
 *
 * What it computes (the per-point Gaussians N(p_i, C_i) of Eq. 19 need, for
 * every query point, its k nearest points in the target cloud and the 3x3
 * covariance of that neighbourhood):
 *
 *   d2(q,p)  = fmaf(dz,dz, fmaf(dy,dy, dx*dx)),  dx = q.x - p.x (binary32,
 *              round to nearest, no contraction) -- the pinned order.
 *   kNN(q)   = the first k target indices under the key (d2, index)
 *              ascending: ties go to the lower index.
 *   C        = (1/k) sum_j (p_j - mu)(p_j - mu)^T, mu = (1/k) sum_j p_j, in
 *              binary64 from the binary32 inputs.
 *   C'       = V diag(1,1,eps) V^T = I - (1 - eps) n n^T, n the unit
 *              eigenvector of the smallest eigenvalue of C (cyclic Jacobi in
 *              binary64); eps < 0 returns C itself.  If tr(C) <= 1e-20 the
 *              neighbourhood is a single point and n := e_z.
 *
 * Two kNN forms: brute force (the definition itself) and a median-split k-d
 * tree whose pruning bound is a proven lower bound on the binary32 d2, so it
 * returns exactly the brute-force answer.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (no fast-math: the
 * d2 order must not be re-associated or fused any further).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------ */
/* The pinned binary32 squared distance.                               */
/* ------------------------------------------------------------------ */
static float sqdist(const float *q, const float *p)
{
    float dx = q[0] - p[0];
    float dy = q[1] - p[1];
    float dz = q[2] - p[2];
    float sx = dx * dx; /* a separate, rounded product */
    return fmaf(dz, dz, fmaf(dy, dy, sx));
}

/* (d2, idx) lexicographic order: does (da, ia) come strictly before (db, ib)? */
static int key_less(float da, int32_t ia, float db, int32_t ib)
{
    if (da < db) return 1;
    if (da > db) return 0;
    return ia < ib;
}

/* A bounded list of the best k entries, kept sorted ascending by key. */
typedef struct {
    int k, n;
    float *d;
    int32_t *i;
} bestlist;

static void best_offer(bestlist *b, float d, int32_t idx)
{
    if (b->n == b->k && !key_less(d, idx, b->d[b->k - 1], b->i[b->k - 1]))
        return;
    int pos = (b->n < b->k) ? b->n : b->k - 1;
    /* shift larger keys one slot towards the end */
    while (pos > 0 && key_less(d, idx, b->d[pos - 1], b->i[pos - 1])) {
        b->d[pos] = b->d[pos - 1];
        b->i[pos] = b->i[pos - 1];
        pos--;
    }
    b->d[pos] = d;
    b->i[pos] = idx;
    if (b->n < b->k) b->n++;
}

/* ------------------------------------------------------------------ */
/* Thread fan-out over query blocks.                                   */
/* ------------------------------------------------------------------ */
typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct {
    range_fn fn;
    void *ctx;
    int64_t lo, hi;
} range_job;

static void *range_thread(void *arg)
{
    range_job *j = (range_job *)arg;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

int oracle_default_threads(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void *ctx)
{
    if (nthreads <= 0) nthreads = oracle_default_threads();
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > n) nthreads = (int)(n > 0 ? n : 1);
    if (nthreads <= 1) {
        fn(ctx, 0, n);
        return;
    }
    pthread_t th[256];
    range_job jobs[256];
    int64_t chunk = (n + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        int64_t lo = t * chunk, hi = lo + chunk;
        if (lo >= n) break;
        if (hi > n) hi = n;
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].lo = lo;
        jobs[t].hi = hi;
        if (pthread_create(&th[t], NULL, range_thread, &jobs[t]) != 0) {
            fn(ctx, lo, hi); /* run inline if a thread cannot start */
            jobs[t].fn = NULL;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; t++)
        if (jobs[t].fn) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ */
/* Brute-force kNN: the definition.                                    */
/* ------------------------------------------------------------------ */
typedef struct {
    const float *q, *p;
    int64_t m;
    int k;
    int32_t *idx;
    float *d2;
} brute_ctx;

static void brute_range(void *vctx, int64_t lo, int64_t hi)
{
    brute_ctx *c = (brute_ctx *)vctx;
    float *bd = (float *)malloc(sizeof(float) * c->k);
    int32_t *bi = (int32_t *)malloc(sizeof(int32_t) * c->k);
    for (int64_t n = lo; n < hi; n++) {
        bestlist b = {c->k, 0, bd, bi};
        const float *q = c->q + 3 * n;
        for (int64_t j = 0; j < c->m; j++)
            best_offer(&b, sqdist(q, c->p + 3 * j), (int32_t)j);
        for (int r = 0; r < c->k; r++) {
            c->idx[n * c->k + r] = bi[r];
            c->d2[n * c->k + r] = bd[r];
        }
    }
    free(bd);
    free(bi);
}

/* q: [n,3] f32, p: [m,3] f32 -> idx [n,k] i32, d2 [n,k] f32.  Returns 0 on
 * success, -1 on bad arguments (k < 1 or k > m). */
int oracle_knn_brute(const float *q, int64_t n, const float *p, int64_t m, int k,
                     int32_t *idx, float *d2, int nthreads)
{
    if (k < 1 || (int64_t)k > m || n < 0) return -1;
    brute_ctx c = {q, p, m, k, idx, d2};
    parallel_for(n, nthreads, brute_range, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Median-split k-d tree.                                              */
/* ------------------------------------------------------------------ */
#define KD_LEAF 8

typedef struct {
    int axis;       /* -1 for a leaf */
    float split;    /* left holds coord <= split, right holds coord >= split */
    int32_t left, right;  /* child node ids */
    int64_t lo, hi;       /* leaf: range into perm */
} kdnode;

typedef struct {
    const float *p; /* caller's points, kept by reference */
    int64_t m;
    int32_t *perm;
    kdnode *nodes;
    int64_t nnodes, cap;
} kdtree;

static float coord(const kdtree *t, int32_t i, int a) { return t->p[3 * (int64_t)i + a]; }

/* Hoare-style quickselect on perm[lo,hi) by coordinate a so that position
 * mid holds the median value, everything before it is <= and everything
 * after it is >=. */
static void kd_select(kdtree *t, int64_t lo, int64_t hi, int64_t mid, int a)
{
    while (hi - lo > 1) {
        float pivot = coord(t, t->perm[lo + (hi - lo) / 2], a);
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (coord(t, t->perm[i], a) < pivot) i++;
            while (coord(t, t->perm[j], a) > pivot) j--;
            if (i <= j) {
                int32_t tmp = t->perm[i];
                t->perm[i] = t->perm[j];
                t->perm[j] = tmp;
                i++;
                j--;
            }
        }
        /* now [lo, j] <= pivot, [i, hi) >= pivot, (j, i) == pivot */
        if (mid <= j)
            hi = j + 1;
        else if (mid >= i)
            lo = i;
        else
            return;
    }
}

static int32_t kd_new_node(kdtree *t)
{
    if (t->nnodes == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->nodes = (kdnode *)realloc(t->nodes, sizeof(kdnode) * t->cap);
    }
    return (int32_t)t->nnodes++;
}

static int32_t kd_build_rec(kdtree *t, int64_t lo, int64_t hi)
{
    int32_t id = kd_new_node(t);
    if (hi - lo <= KD_LEAF) {
        kdnode leaf = {-1, 0.0f, -1, -1, lo, hi};
        t->nodes[id] = leaf;
        return id;
    }
    float mn[3], mx[3];
    for (int a = 0; a < 3; a++) mn[a] = mx[a] = coord(t, t->perm[lo], a);
    for (int64_t i = lo + 1; i < hi; i++)
        for (int a = 0; a < 3; a++) {
            float v = coord(t, t->perm[i], a);
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    int axis = 0;
    for (int a = 1; a < 3; a++)
        if (mx[a] - mn[a] > mx[axis] - mn[axis]) axis = a;
    int64_t mid = lo + (hi - lo) / 2;
    kd_select(t, lo, hi, mid, axis);
    float split = coord(t, t->perm[mid], axis);
    /* left = [lo, mid), right = [mid, hi): left coords <= split <= right */
    int32_t l = kd_build_rec(t, lo, mid);
    int32_t r = kd_build_rec(t, mid, hi);
    kdnode in = {axis, split, l, r, lo, hi};
    t->nodes[id] = in;
    return id;
}

void *oracle_kdtree_build(const float *p, int64_t m)
{
    if (m < 1) return NULL;
    kdtree *t = (kdtree *)calloc(1, sizeof(kdtree));
    t->p = p;
    t->m = m;
    t->perm = (int32_t *)malloc(sizeof(int32_t) * m);
    for (int64_t i = 0; i < m; i++) t->perm[i] = (int32_t)i;
    kd_build_rec(t, 0, m);
    return t;
}

void oracle_kdtree_free(void *vt)
{
    kdtree *t = (kdtree *)vt;
    if (!t) return;
    free(t->perm);
    free(t->nodes);
    free(t);
}

static void kd_search(const kdtree *t, int32_t id, const float *q, bestlist *b)
{
    const kdnode *nd = &t->nodes[id];
    if (nd->axis < 0) {
        for (int64_t i = nd->lo; i < nd->hi; i++) {
            int32_t j = t->perm[i];
            best_offer(b, sqdist(q, t->p + 3 * (int64_t)j), j);
        }
        return;
    }
    float qa = q[nd->axis];
    int32_t near = (qa <= nd->split) ? nd->left : nd->right;
    int32_t far = (qa <= nd->split) ? nd->right : nd->left;
    kd_search(t, near, q, b);
    /* Every far-side point p has |fl(q_a - p_a)| >= |fl(q_a - split)| by
     * monotone rounding, and the binary32 d2 is a rounded sum of
     * non-negative terms, so fl(s*s) bounds its d2 from below.  Ties must
     * still be visited (a lower index may win), hence <=. */
    float s = qa - nd->split;
    float lb = s * s;
    if (b->n < b->k || lb <= b->d[b->k - 1]) kd_search(t, far, q, b);
}

typedef struct {
    const kdtree *t;
    const float *q;
    int k;
    int32_t *idx;
    float *d2;
} kdq_ctx;

static void kdq_range(void *vctx, int64_t lo, int64_t hi)
{
    kdq_ctx *c = (kdq_ctx *)vctx;
    float *bd = (float *)malloc(sizeof(float) * c->k);
    int32_t *bi = (int32_t *)malloc(sizeof(int32_t) * c->k);
    for (int64_t n = lo; n < hi; n++) {
        bestlist b = {c->k, 0, bd, bi};
        kd_search(c->t, 0, c->q + 3 * n, &b);
        for (int r = 0; r < c->k; r++) {
            c->idx[n * c->k + r] = bi[r];
            c->d2[n * c->k + r] = bd[r];
        }
    }
    free(bd);
    free(bi);
}

int oracle_kdtree_knn(void *vt, const float *q, int64_t n, int k, int32_t *idx, float *d2,
                      int nthreads)
{
    kdtree *t = (kdtree *)vt;
    if (!t || k < 1 || (int64_t)k > t->m || n < 0) return -1;
    kdq_ctx c = {t, q, k, idx, d2};
    parallel_for(n, nthreads, kdq_range, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations.        */
/* ------------------------------------------------------------------ */
/* a6 = (xx, xy, xz, yy, yz, zz).  On return w[0..2] are the eigenvalues
 * (ascending) and V (row-major 3x3) holds the matching unit eigenvectors as
 * its COLUMNS.  Each rotation zeroes one off-diagonal entry a_pq exactly
 * (Jacobi's method, Golub & Van Loan sec. 8.5); sweeps repeat until the
 * off-diagonal mass is negligible. */
void oracle_eig_sym3(const double *a6, double *w, double *V)
{
    double A[3][3] = {{a6[0], a6[1], a6[2]}, {a6[1], a6[3], a6[4]}, {a6[2], a6[4], a6[5]}};
    double Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 64; sweep++) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-36 * diag) break;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                double apq = A[p][q];
                if (apq == 0.0) continue;
                /* choose the rotation angle so that the new a_pq is zero */
                double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                /* A <- J^T A J with J the (p,q) plane rotation */
                for (int r = 0; r < 3; r++) {
                    double arp = A[r][p], arq = A[r][q];
                    A[r][p] = c * arp - s * arq;
                    A[r][q] = s * arp + c * arq;
                }
                for (int r = 0; r < 3; r++) {
                    double apr = A[p][r], aqr = A[q][r];
                    A[p][r] = c * apr - s * aqr;
                    A[q][r] = s * apr + c * aqr;
                }
                for (int r = 0; r < 3; r++) {
                    double qrp = Q[r][p], qrq = Q[r][q];
                    Q[r][p] = c * qrp - s * qrq;
                    Q[r][q] = s * qrp + c * qrq;
                }
            }
    }
    /* sort ascending, permuting eigenvector columns along */
    int order[3] = {0, 1, 2};
    for (int i = 0; i < 3; i++)
        for (int j = i + 1; j < 3; j++)
            if (A[order[j]][order[j]] < A[order[i]][order[i]]) {
                int tmp = order[i];
                order[i] = order[j];
                order[j] = tmp;
            }
    for (int i = 0; i < 3; i++) {
        w[i] = A[order[i]][order[i]];
        for (int r = 0; r < 3; r++) V[3 * r + i] = Q[r][order[i]];
    }
}

/* ------------------------------------------------------------------ */
/* Neighbourhood covariance in binary64.                               */
/* ------------------------------------------------------------------ */
/* One neighbourhood: points p[idx[j]], j < k.  Writes the 6 upper-triangle
 * entries (xx, xy, xz, yy, yz, zz) of C (eps < 0) or of C' (eps >= 0). */
void oracle_cov_one(const float *p, const int32_t *nb, int k, double eps, double *out)
{
    double mu[3] = {0, 0, 0};
    for (int j = 0; j < k; j++)
        for (int a = 0; a < 3; a++) mu[a] += (double)p[3 * (int64_t)nb[j] + a];
    for (int a = 0; a < 3; a++) mu[a] /= (double)k;
    double C[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < k; j++) {
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = (double)p[3 * (int64_t)nb[j] + a] - mu[a];
        C[0] += d[0] * d[0];
        C[1] += d[0] * d[1];
        C[2] += d[0] * d[2];
        C[3] += d[1] * d[1];
        C[4] += d[1] * d[2];
        C[5] += d[2] * d[2];
    }
    for (int e = 0; e < 6; e++) C[e] /= (double)k;
    if (eps < 0) {
        memcpy(out, C, sizeof(C));
        return;
    }
    double n[3] = {0, 0, 1};
    if (C[0] + C[3] + C[5] > 1e-20) {
        double w[3], V[9];
        oracle_eig_sym3(C, w, V);
        for (int r = 0; r < 3; r++) n[r] = V[3 * r + 0];
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int r = 0; r < 3; r++) n[r] /= nn;
    }
    double f = 1.0 - eps;
    out[0] = 1.0 - f * n[0] * n[0];
    out[1] = -f * n[0] * n[1];
    out[2] = -f * n[0] * n[2];
    out[3] = 1.0 - f * n[1] * n[1];
    out[4] = -f * n[1] * n[2];
    out[5] = 1.0 - f * n[2] * n[2];
}

typedef struct {
    const float *p;
    const int32_t *idx;
    int k;
    double eps;
    double *cov;
} cov_ctx;

static void cov_range(void *vctx, int64_t lo, int64_t hi)
{
    cov_ctx *c = (cov_ctx *)vctx;
    for (int64_t n = lo; n < hi; n++)
        oracle_cov_one(c->p, c->idx + n * c->k, c->k, c->eps, c->cov + 6 * n);
}

/* p: [m,3] f32 target, idx: [n,k] neighbour rows -> cov [n,6] f64. */
int oracle_cov(const float *p, int64_t m, const int32_t *idx, int64_t n, int k, double eps,
               double *cov, int nthreads)
{
    if (k < 1 || n < 0) return -1;
    for (int64_t i = 0; i < n * (int64_t)k; i++)
        if (idx[i] < 0 || (int64_t)idx[i] >= m) return -2;
    cov_ctx c = {p, idx, k, eps, cov};
    parallel_for(n, nthreads, cov_range, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* GICP linearisation (Eq. 18-20), one Gauss-Newton step.              */
/* ------------------------------------------------------------------ */
/* pose = R (row-major 3x3) then t (3), binary32.  Every source point p is
 * moved to p' = R p + t in binary32 with the pinned order
 *     p'_a = fmaf(R_a2, p_z, fmaf(R_a1, p_y, fmaf(R_a0, p_x, t_a)))
 * and matched to its nearest map point q (d2 and ties as in the kNN above).
 * The pair is an inlier when p' is finite and d2 <= fl(max_dist^2).
 *
 * In binary64, with the residual d = q - p' (Eq. 18) and the combined
 * covariance S = C_q + R C_p R^T (Eq. 19; the printed form of that sum is
 * garbled, this is the standard GICP one), Omega = S^-1 and the step sums
 *     H = sum J^T Omega J,  b = sum J^T Omega d,  E = sum d^T Omega d
 * over the inliers whose S has a positive determinant, with
 * J = [ [p']_x , -I ] the derivative of d under the left perturbation
 * T <- exp(xi^) T, xi = (omega, v): T p ~ p' + omega x p' + v.
 * Minimising sum (d + J xi)^T Omega (d + J xi) gives H xi = -b.
 *
 * out (29 doubles): H upper triangle row by row (21), b (6), E, the number
 * of pairs summed.  corr (optional, [n]): the map index of each inlier
 * pair, -1 for the others. */
void oracle_gicp_transform(const float *pose, const float *src, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; i++) {
        const float *p = src + 3 * i;
        for (int a = 0; a < 3; a++)
            out[3 * i + a] =
                fmaf(pose[3 * a + 2], p[2], fmaf(pose[3 * a + 1], p[1], fmaf(pose[3 * a + 0], p[0], pose[9 + a])));
    }
}

static void sym6_to_mat(const float *c, double M[3][3])
{
    M[0][0] = c[0]; M[0][1] = c[1]; M[0][2] = c[2];
    M[1][0] = c[1]; M[1][1] = c[3]; M[1][2] = c[4];
    M[2][0] = c[2]; M[2][1] = c[4]; M[2][2] = c[5];
}

/* Inverse of a symmetric 3x3 as adjugate / determinant; returns 0 (and
 * leaves O alone) when the determinant is not positive. */
static int inv_sym3(double S[3][3], double O[3][3])
{
    const double a00 = S[1][1] * S[2][2] - S[1][2] * S[2][1];
    const double a01 = S[0][2] * S[2][1] - S[0][1] * S[2][2];
    const double a02 = S[0][1] * S[1][2] - S[0][2] * S[1][1];
    const double a11 = S[0][0] * S[2][2] - S[0][2] * S[2][0];
    const double a12 = S[0][2] * S[1][0] - S[0][0] * S[1][2];
    const double a22 = S[0][0] * S[1][1] - S[0][1] * S[1][0];
    const double det = S[0][0] * a00 + S[1][0] * a01 + S[2][0] * a02;
    if (!(det > 0)) return 0;
    O[0][0] = a00 / det; O[0][1] = a01 / det; O[0][2] = a02 / det;
    O[1][0] = a01 / det; O[1][1] = a11 / det; O[1][2] = a12 / det;
    O[2][0] = a02 / det; O[2][1] = a12 / det; O[2][2] = a22 / det;
    return 1;
}

int oracle_gicp_linearize(void *vt, const float *map_cov, const float *src, int64_t n, const float *src_cov,
                          const float *pose, float max_dist, double *out, int32_t *corr, int nthreads)
{
    kdtree *t = (kdtree *)vt;
    if (!t || n < 0 || !(max_dist >= 0)) return -1;
    const int64_t nn_ = n > 0 ? n : 1;
    float *moved = (float *)malloc(sizeof(float) * 3 * nn_);
    float *fin = (float *)malloc(sizeof(float) * 3 * nn_);
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * nn_);
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * nn_);
    float *nd = (float *)malloc(sizeof(float) * nn_);
    oracle_gicp_transform(pose, src, n, moved);
    /* nearest map point of every finite moved point */
    int64_t nf = 0;
    for (int64_t i = 0; i < n; i++) {
        if (corr) corr[i] = -1;
        if (isfinite(moved[3 * i]) && isfinite(moved[3 * i + 1]) && isfinite(moved[3 * i + 2])) {
            memcpy(fin + 3 * nf, moved + 3 * i, 3 * sizeof(float));
            pos[nf++] = i;
        }
    }
    if (nf > 0) oracle_kdtree_knn(vt, fin, nf, 1, nb, nd, nthreads);
    const float max_d2 = max_dist * max_dist;
    double R[3][3];
    for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) R[a][c] = pose[3 * a + c];
    double H[6][6] = {{0}}, b[6] = {0}, E = 0, pairs = 0;
    for (int64_t f = 0; f < nf; f++) {
        if (!(nd[f] <= max_d2)) continue;
        const int64_t i = pos[f];
        if (corr) corr[i] = nb[f];
        const float *q = t->p + 3 * (int64_t)nb[f];
        const double pp[3] = {fin[3 * f], fin[3 * f + 1], fin[3 * f + 2]};
        const double d[3] = {(double)q[0] - pp[0], (double)q[1] - pp[1], (double)q[2] - pp[2]};
        double Cq[3][3], Cp[3][3], S[3][3], O[3][3];
        sym6_to_mat(map_cov + 6 * (int64_t)nb[f], Cq);
        sym6_to_mat(src_cov + 6 * i, Cp);
        /* S = Cq + R Cp R^T */
        for (int a = 0; a < 3; a++)
            for (int c = 0; c < 3; c++) {
                double s = 0;
                for (int e = 0; e < 3; e++)
                    for (int g = 0; g < 3; g++) s += R[a][e] * Cp[e][g] * R[c][g];
                S[a][c] = Cq[a][c] + s;
            }
        if (!inv_sym3(S, O)) continue;
        const double J[3][6] = {{0, -pp[2], pp[1], -1, 0, 0},
                                {pp[2], 0, -pp[0], 0, -1, 0},
                                {-pp[1], pp[0], 0, 0, 0, -1}};
        for (int r = 0; r < 6; r++) {
            for (int c = r; c < 6; c++)
                for (int a = 0; a < 3; a++)
                    for (int e = 0; e < 3; e++) H[r][c] += J[a][r] * O[a][e] * J[e][c];
            for (int a = 0; a < 3; a++)
                for (int e = 0; e < 3; e++) b[r] += J[a][r] * O[a][e] * d[e];
        }
        for (int a = 0; a < 3; a++)
            for (int e = 0; e < 3; e++) E += d[a] * O[a][e] * d[e];
        pairs += 1;
    }
    int w = 0;
    for (int r = 0; r < 6; r++)
        for (int c = r; c < 6; c++) out[w++] = H[r][c];
    for (int r = 0; r < 6; r++) out[w++] = b[r];
    out[w++] = E;
    out[w++] = pairs;
    free(moved);
    free(fin);
    free(pos);
    free(nb);
    free(nd);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Kernel-descriptor weighted covariance (Sec. III-C1, Table I).       */
/* ------------------------------------------------------------------ */
/* The paper computes the per-point covariance "using the kernel
 * descriptors" of Table I without stating where the kernel enters; this
 * reads it as a weight on every neighbour, w_j = K(q, p_j), in a weighted
 * mean and weighted second moments:
 *     W = sum w_j,  mu = sum w_j p_j / W,
 *     C = sum w_j (p_j - mu)(p_j - mu)^T / W,
 * then the same plane regularisation as oracle_cov_one (eps >= 0).  The
 * kernels, with x = q and y = p_j:
 *     1 RBF         exp(-|x - y|^2 sigma)
 *     2 Gaussian    exp(-|x - y|^2 / (2 sigma^2))
 *     3 Polynomial  (alpha <x', y'> + c)^d
 *     4 HI          sum_i min(x'_i, y'_i) / sum_i x'_i
 *     5 Laplacian   exp(-|x - y| / sigma)
 * where x' = x - o, y' = y - o are coordinates relative to o, the target's
 * bounding-box minimum (Polynomial and HI depend on absolute coordinates;
 * this fixes their origin to the map's own).  Everything is binary64 from
 * the binary32 inputs.  A row whose total weight is not positive and finite
 * is NaN. */
static double kd_weight(int type, const double *x, const double *y, const double *o, double sigma,
                        double alpha, double c, double d)
{
    double r2 = 0, dot = 0, mn = 0, sx = 0;
    for (int a = 0; a < 3; a++) {
        const double e = x[a] - y[a];
        r2 += e * e;
        const double xa = x[a] - o[a], ya = y[a] - o[a];
        dot += xa * ya;
        mn += xa < ya ? xa : ya;
        sx += xa;
    }
    switch (type) {
    case 1: return exp(-r2 * sigma);
    case 2: return exp(-r2 / (2.0 * sigma * sigma));
    case 3: return pow(alpha * dot + c, d);
    case 4: return mn / sx;
    case 5: return exp(-sqrt(r2) / sigma);
    }
    return 1.0;
}

void oracle_cov_weighted_one(const float *p, const int32_t *nb, int k, const float *q, int type,
                             const double *prm, const double *o, double eps, double *out)
{
    double x[3] = {q[0], q[1], q[2]};
    double W = 0, mu[3] = {0, 0, 0};
    double *w = (double *)malloc(sizeof(double) * k);
    for (int j = 0; j < k; j++) {
        const double y[3] = {p[3 * (int64_t)nb[j]], p[3 * (int64_t)nb[j] + 1], p[3 * (int64_t)nb[j] + 2]};
        w[j] = kd_weight(type, x, y, o, prm[0], prm[1], prm[2], prm[3]);
        W += w[j];
        for (int a = 0; a < 3; a++) mu[a] += w[j] * y[a];
    }
    if (!(W > 0) || !isfinite(W)) {
        for (int e = 0; e < 6; e++) out[e] = NAN;
        free(w);
        return;
    }
    for (int a = 0; a < 3; a++) mu[a] /= W;
    double C[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < k; j++) {
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = (double)p[3 * (int64_t)nb[j] + a] - mu[a];
        C[0] += w[j] * d[0] * d[0];
        C[1] += w[j] * d[0] * d[1];
        C[2] += w[j] * d[0] * d[2];
        C[3] += w[j] * d[1] * d[1];
        C[4] += w[j] * d[1] * d[2];
        C[5] += w[j] * d[2] * d[2];
    }
    free(w);
    for (int e = 0; e < 6; e++) C[e] /= W;
    if (eps < 0) {
        memcpy(out, C, sizeof(C));
        return;
    }
    double n[3] = {0, 0, 1};
    if (C[0] + C[3] + C[5] > 1e-20) {
        double ev[3], V[9];
        oracle_eig_sym3(C, ev, V);
        for (int r = 0; r < 3; r++) n[r] = V[3 * r + 0];
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int r = 0; r < 3; r++) n[r] /= nn;
    }
    double f = 1.0 - eps;
    out[0] = 1.0 - f * n[0] * n[0];
    out[1] = -f * n[0] * n[1];
    out[2] = -f * n[0] * n[2];
    out[3] = 1.0 - f * n[1] * n[1];
    out[4] = -f * n[1] * n[2];
    out[5] = 1.0 - f * n[2] * n[2];
}

/* q: [n,3], idx: [n,k] rows into p: [m,3]; prm = (sigma, alpha, c, d);
 * o = the target's bounding-box minimum.  Returns -1 / -2 as oracle_cov. */
int oracle_cov_weighted(const float *p, int64_t m, const float *q, const int32_t *idx, int64_t n, int k,
                        double eps, int type, const double *prm, const double *o, double *cov)
{
    if (k < 1 || n < 0 || type < 0 || type > 5) return -1;
    for (int64_t i = 0; i < n * (int64_t)k; i++)
        if (idx[i] < 0 || (int64_t)idx[i] >= m) return -2;
    for (int64_t i = 0; i < n; i++)
        oracle_cov_weighted_one(p, idx + i * k, k, q + 3 * i, type, prm, o, eps, cov + 6 * i);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ground filter by 2-D voting and wall clustering (Sec. III-D, Eq.    */
/* 24-30).                                                             */
/* ------------------------------------------------------------------ */
/* Points are in the vehicle body frame (x forward, y left).  Steps, in the
 * paper's order:
 *  1. voxel filter: voxel (i,j,k) = floor(fl(p * fl(1/v))) per axis; points
 *     whose voxel lies outside -2^(b-1) <= i <= 2^(b-1) - 2 (b = bxy for i, j
 *     and bz for k, sized to hold the configured range) or that are not
 *     finite are dropped.  Voxels are
 *     numbered in ascending key order, key = (i+o) | (j+o) << bxy |
 *     (k+oz) << 2 bxy; each voxelised point is the centroid of its points,
 *     summed in binary64 in input order, divided by the count and rounded to
 *     binary32 (Eq. 24: one representative per voxel);
 *  2. vote: each voxel votes for the 2-D cell floor(fl(c_x * fl(1/g))),
 *     floor(fl(c_y * fl(1/g))) of its centroid; a voxel is a vertical
 *     feature when its cell holds more than min_votes voxels, ground
 *     otherwise (Eq. 25 and the hyper-parameter comparison);
 *  3. Euclidean clustering of the vertical voxels: two are linked when the
 *     pinned binary32 d2 of their centroids is <= fl(tol * tol); clusters
 *     are the connected components, labelled by their smallest voxel index
 *     (Eq. 26, read as the usual single-linkage tree clustering the text
 *     names);
 *  4. the wall: among clusters of at least min_cluster voxels on the right
 *     (fl(min y + max y) < 0), the longest, length = fl(max x - min x);
 *     ties to the smaller label (Eq. 27, H = the cluster's length);
 *  5. y = b0 + b1 x + b2 x^2 by least squares over the wall's centroids,
 *     normal equations in binary64 (Eq. 28); d_w = b0 is y at the vehicle
 *     origin x = 0 (Eq. 29); b1, b2 are the path coefficients (Eq. 30).
 * Outputs per voxel (in key order): centroid, vertical flag, label (-1 for
 * ground).  Returns the number of voxels, or a negative code. */
typedef struct {
    uint64_t key;
    int64_t idx;
} keyidx;

static int keyidx_cmp(const void *a, const void *b)
{
    const keyidx *x = (const keyidx *)a, *y = (const keyidx *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int64_t uf_find(int64_t *par, int64_t a)
{
    while (par[a] != a) a = par[a];
    return a;
}

static int bits_to_hold(int64_t n)
{
    int b = 1;
    while (((int64_t)1 << b) < n) b++;
    return b;
}

int64_t oracle_wall_detect(const float *pts, int64_t n, float voxel, float cell2d, int min_votes, float tol,
                           int min_cluster, float max_range, float max_height, float *cent, int32_t *vertical,
                           int64_t *label, int64_t *wall_label, double *beta, int64_t *wall_count)
{
    if (n < 0 || !(voxel > 0) || !(cell2d > 0) || !(tol > 0) || !(max_range > 0) || !(max_height > 0)) return -1;
    const float inv_v = 1.0f / voxel, inv_g = 1.0f / cell2d;
    const int64_t rxy = (int64_t)ceil(max_range / voxel) + 1, rz = (int64_t)ceil(max_height / voxel) + 1;
    const int bxy = bits_to_hold(2 * rxy), bz = bits_to_hold(2 * rz);
    if (2 * bxy + bz > 63) return -1;
    const int64_t oxy = (int64_t)1 << (bxy - 1), oz = (int64_t)1 << (bz - 1);
    keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * (n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        const float *p = pts + 3 * i;
        if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) continue;
        const double fi = floor((double)(p[0] * inv_v)), fj = floor((double)(p[1] * inv_v)),
                     fk = floor((double)(p[2] * inv_v));
        /* kept: -o <= i <= o - 2, so a field never reaches all ones (that key
         * marks a dropped point) */
        if (fi < -(double)oxy || fi > (double)(oxy - 2) || fj < -(double)oxy || fj > (double)(oxy - 2) ||
            fk < -(double)oz || fk > (double)(oz - 2))
            continue;
        const uint64_t ci = (uint64_t)((int64_t)fi + oxy), cj = (uint64_t)((int64_t)fj + oxy),
                       ck = (uint64_t)((int64_t)fk + oz);
        ki[m].key = ci | (cj << bxy) | (ck << (2 * bxy));
        ki[m].idx = i;
        m++;
    }
    qsort(ki, (size_t)m, sizeof(keyidx), keyidx_cmp);
    /* 1. voxel centroids */
    int64_t nv = 0;
    for (int64_t s = 0; s < m;) {
        int64_t e = s;
        double sx = 0, sy = 0, sz = 0;
        while (e < m && ki[e].key == ki[s].key) {
            const float *p = pts + 3 * ki[e].idx;
            sx += p[0];
            sy += p[1];
            sz += p[2];
            e++;
        }
        const double c = (double)(e - s);
        cent[3 * nv] = (float)(sx / c);
        cent[3 * nv + 1] = (float)(sy / c);
        cent[3 * nv + 2] = (float)(sz / c);
        nv++;
        s = e;
    }
    free(ki);
    /* 2. votes per 2-D cell (sorted cell keys) */
    keyidx *ck = (keyidx *)malloc(sizeof(keyidx) * (nv > 0 ? nv : 1));
    for (int64_t v = 0; v < nv; v++) {
        const int64_t u = (int64_t)floor((double)(cent[3 * v] * inv_g));
        const int64_t w = (int64_t)floor((double)(cent[3 * v + 1] * inv_g));
        ck[v].key = ((uint64_t)(u + ((int64_t)1 << 31)) << 32) | (uint64_t)(w + ((int64_t)1 << 31));
        ck[v].idx = v;
    }
    qsort(ck, (size_t)nv, sizeof(keyidx), keyidx_cmp);
    for (int64_t s = 0; s < nv;) {
        int64_t e = s;
        while (e < nv && ck[e].key == ck[s].key) e++;
        for (int64_t t = s; t < e; t++) vertical[ck[t].idx] = (e - s) > min_votes;
        s = e;
    }
    free(ck);
    /* 3. clustering of the vertical voxels: brute force pairs, union-find
     * hooking the larger root under the smaller */
    int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (nv > 0 ? nv : 1));
    for (int64_t v = 0; v < nv; v++) par[v] = v;
    const float tol2 = tol * tol;
    for (int64_t a = 0; a < nv; a++) {
        if (!vertical[a]) continue;
        for (int64_t b = a + 1; b < nv; b++) {
            if (!vertical[b]) continue;
            if (sqdist(cent + 3 * a, cent + 3 * b) <= tol2) {
                int64_t ra = uf_find(par, a), rb = uf_find(par, b);
                if (ra != rb) {
                    if (ra < rb) par[rb] = ra;
                    else par[ra] = rb;
                }
            }
        }
    }
    for (int64_t v = 0; v < nv; v++) label[v] = vertical[v] ? uf_find(par, v) : -1;
    free(par);
    /* 4. the wall */
    float *mnx = (float *)malloc(sizeof(float) * (nv > 0 ? nv : 1));
    float *mxx = (float *)malloc(sizeof(float) * (nv > 0 ? nv : 1));
    float *mny = (float *)malloc(sizeof(float) * (nv > 0 ? nv : 1));
    float *mxy = (float *)malloc(sizeof(float) * (nv > 0 ? nv : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)(nv > 0 ? nv : 1), sizeof(int64_t));
    for (int64_t v = 0; v < nv; v++) {
        if (label[v] < 0) continue;
        const int64_t L = label[v];
        const float x = cent[3 * v], y = cent[3 * v + 1];
        if (cnt[L] == 0) {
            mnx[L] = mxx[L] = x;
            mny[L] = mxy[L] = y;
        } else {
            if (x < mnx[L]) mnx[L] = x;
            if (x > mxx[L]) mxx[L] = x;
            if (y < mny[L]) mny[L] = y;
            if (y > mxy[L]) mxy[L] = y;
        }
        cnt[L]++;
    }
    int64_t best = -1;
    float best_len = -1.0f;
    for (int64_t L = 0; L < nv; L++) {
        if (cnt[L] < min_cluster || cnt[L] == 0) continue;
        if (!(mny[L] + mxy[L] < 0.0f)) continue;
        const float len = mxx[L] - mnx[L];
        if (len > best_len) {
            best_len = len;
            best = L;
        }
    }
    *wall_label = best;
    *wall_count = best >= 0 ? cnt[best] : 0;
    /* 5. least squares y = b0 + b1 x + b2 x^2 */
    beta[0] = beta[1] = beta[2] = NAN;
    if (best >= 0) {
        double A[3][3] = {{0}}, r[3] = {0};
        for (int64_t v = 0; v < nv; v++) {
            if (label[v] != best) continue;
            const double x = cent[3 * v], y = cent[3 * v + 1];
            const double f[3] = {1.0, x, x * x};
            for (int a = 0; a < 3; a++) {
                for (int b = 0; b < 3; b++) A[a][b] += f[a] * f[b];
                r[a] += f[a] * y;
            }
        }
        /* Gaussian elimination with partial pivoting */
        double M[3][4];
        for (int a = 0; a < 3; a++) {
            for (int b = 0; b < 3; b++) M[a][b] = A[a][b];
            M[a][3] = r[a];
        }
        int ok = 1;
        for (int c = 0; c < 3 && ok; c++) {
            int piv = c;
            for (int a = c + 1; a < 3; a++)
                if (fabs(M[a][c]) > fabs(M[piv][c])) piv = a;
            if (!(fabs(M[piv][c]) > 0)) {
                ok = 0;
                break;
            }
            for (int b = 0; b < 4; b++) {
                double t = M[c][b];
                M[c][b] = M[piv][b];
                M[piv][b] = t;
            }
            for (int a = 0; a < 3; a++) {
                if (a == c) continue;
                const double f = M[a][c] / M[c][c];
                for (int b = c; b < 4; b++) M[a][b] -= f * M[c][b];
            }
        }
        if (ok)
            for (int a = 0; a < 3; a++) beta[a] = M[a][3] / M[a][a];
    }
    free(mnx);
    free(mxx);
    free(mny);
    free(mxy);
    free(cnt);
    return nv;
}
