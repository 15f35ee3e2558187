/*
 * FP64 CPU oracle for the balanced-tree adaptive FMM in 3D
 * (Bull & Engblom, "Distributed and Adaptive Fast Multipole Method in
 * Three Dimensions", arXiv:2002.04894).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it. It shares no code, header or table with the
 * CUDA implementation.
 *
 * It is deliberately plain and slow: every stage is the textbook formula or
 * the paper's algorithm written out as nested loops in double precision,
 * with double complex arithmetic. Compile with -ffp-contract=off so that no
 * multiply-add is fused (the tree geometry and the theta-criterion must be
 * reproducible to the bit).
 *
 * Stages, in the order of Algorithm 1:
 *   Tree  (Algorithm 2, Sec. 2.1.2)  median-plane bisection, fixed levels
 *   Lists (Eq. 2.2, Sec. 2.1.1)      theta-criterion connectivity
 *   P2M, M2M (Algorithm 1)           multipole expansions, upward pass
 *   M2L, L2L (Algorithm 3)           local expansions, downward pass
 *   L2P, P2P (Algorithm 4)           evaluation at the leaf points
 * plus the exact pairwise sum of Eq. 2.1 that the method approximates.
 *
 * Readings where the paper is silent (each is listed with its reason in
 * the design notes of the repository):
 *  - a "level" is one binary bisection; a box splits on the longest axis of
 *    its cell (ties: x before y before z);
 *  - keys are (coordinate on that axis, original index); the left child
 *    gets the floor(n/2) smallest keys; both children keep ascending
 *    original-index order;
 *  - split plane s = 0.5*(max_left + min_right); one point: s = its
 *    coordinate; no point: s = cell midpoint; for eta < 1 the plane is
 *    eta*s + (1-eta)*midpoint and the left child takes the points strictly
 *    below it (Sec. 2.1.2's adaptivity parameter);
 *  - root cell = tight bounding box; box centre = cell midpoint; radius =
 *    half the cell diagonal (the default), or, with `tight` set, the
 *    midpoint and half diagonal of the bounding box of the box's own points,
 *    the radius never below 2^-10 of the cell's (a box of one point keeps a
 *    positive size; an empty box keeps its cell midpoint); the cells still
 *    decide the splits;
 *  - weak iff theta > 0, d > 0 and R + theta*r <= theta*d;
 *  - M2L at every level that has weak pairs (leaf level included);
 *  - the paper's octree levels (8 children per box) are `step` = 3
 *    successive bisections per FMM level; connectivity, M2M, M2L and L2L
 *    then act only on every step-th bisection level (step 1: every level);
 *  - coincident points (r^2 == 0) are skipped in every pairwise sum.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Solid harmonics (Sec. 2.1: spherical-harmonic expansions)           */
/* ------------------------------------------------------------------ */

/* Index of coefficient (n, m), 0 <= m <= n, in a packed triangle. */
static int tri(int n, int m) { return n * (n + 1) / 2 + m; }

int orc_ncoef(int p) { return (p + 1) * (p + 2) / 2; }

/*
 * Regular solid harmonic R_n^m(x) = r^n P_n^m(cos t) e^{i m phi} / (n+m)!
 * for 0 <= m <= n <= p, with P_n^m the associated Legendre function without
 * the Condon-Shortley phase. Written from the Legendre recurrences:
 *   R_m^m     = (x + i y) / (2m) * R_{m-1}^{m-1}
 *   R_{m+1}^m = z R_m^m
 *   R_n^m     = ((2n-1) z R_{n-1}^m - r^2 R_{n-2}^m) / ((n-m)(n+m)).
 */
void orc_regular(const double x[3], int p, cplx *R)
{
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    cplx w = x[0] + I * x[1];
    R[tri(0, 0)] = 1.0;
    for (int m = 0; m <= p; m++) {
        if (m > 0)
            R[tri(m, m)] = w / (2.0 * m) * R[tri(m - 1, m - 1)];
        if (m + 1 <= p)
            R[tri(m + 1, m)] = x[2] * R[tri(m, m)];
        for (int n = m + 2; n <= p; n++)
            R[tri(n, m)] = ((2.0 * n - 1.0) * x[2] * R[tri(n - 1, m)]
                            - r2 * R[tri(n - 2, m)])
                           / ((double)(n - m) * (double)(n + m));
    }
}

/*
 * Irregular solid harmonic I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m phi} / r^{n+1}
 * for 0 <= m <= n <= p (x != 0). Recurrences:
 *   I_0^0     = 1/r
 *   I_m^m     = (2m-1)(x + i y)/r^2 * I_{m-1}^{m-1}
 *   I_{m+1}^m = (2m+1) z / r^2 * I_m^m
 *   I_n^m     = ((2n-1) z I_{n-1}^m - (n-1+m)(n-1-m) I_{n-2}^m) / r^2.
 */
void orc_irregular(const double x[3], int p, cplx *Ir)
{
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    cplx w = x[0] + I * x[1];
    Ir[tri(0, 0)] = 1.0 / sqrt(r2);
    for (int m = 0; m <= p; m++) {
        if (m > 0)
            Ir[tri(m, m)] = (2.0 * m - 1.0) * w / r2 * Ir[tri(m - 1, m - 1)];
        if (m + 1 <= p)
            Ir[tri(m + 1, m)] = (2.0 * m + 1.0) * x[2] / r2 * Ir[tri(m, m)];
        for (int n = m + 2; n <= p; n++)
            Ir[tri(n, m)] = ((2.0 * n - 1.0) * x[2] * Ir[tri(n - 1, m)]
                             - (double)(n - 1 + m) * (double)(n - 1 - m)
                                   * Ir[tri(n - 2, m)])
                            / r2;
    }
}

/*
 * Signed-order views. Upsilon_n^m = (-1)^m R_n^m and Theta_n^m = (-1)^m I_n^m
 * for m >= 0, Upsilon_n^{-m} = conj(R_n^m), Theta_n^{-m} = conj(I_n^m). With
 * these, 1/|x - y| = sum_{n,m} conj(Upsilon_n^m(y)) Theta_n^m(x) (|y| < |x|),
 * Upsilon_n^m(a + b) = sum_{k,l} Upsilon_k^l(a) Upsilon_{n-k}^{m-l}(b), and
 * Theta_n^m(x - y) = sum_{k,l} conj(Upsilon_k^l(y)) Theta_{n+k}^{m+l}(x).
 */
static cplx signed_view(const cplx *H, int n, int m)
{
    if (n < 0 || m > n || -m > n)
        return 0.0;
    if (m >= 0)
        return (m & 1) ? -H[tri(n, m)] : H[tri(n, m)];
    return conj(H[tri(n, -m)]);
}

/*
 * Expansion coefficients of a real charge distribution obey
 * C_n^{-m} = (-1)^m conj(C_n^m); only m >= 0 is stored.
 */
static cplx coef(const cplx *C, int n, int m)
{
    if (n < 0 || m > n || -m > n)
        return 0.0;
    if (m >= 0)
        return C[tri(n, m)];
    return ((-m) & 1) ? -conj(C[tri(n, -m)]) : conj(C[tri(n, -m)]);
}

/* ------------------------------------------------------------------ */
/* Expansion operators (Algorithm 1, Algorithm 3, Algorithm 4)         */
/* ------------------------------------------------------------------ */

/* P2M: M_n^m += sum_j q_j conj(Upsilon_n^m(x_j - c)). Points are n x 3. */
void orc_p2m(int64_t np, const double *x, const double *q, const double c[3],
             int p, cplx *M)
{
    cplx *R = malloc(sizeof(cplx) * orc_ncoef(p));
    for (int64_t j = 0; j < np; j++) {
        double d[3] = {x[3 * j] - c[0], x[3 * j + 1] - c[1], x[3 * j + 2] - c[2]};
        orc_regular(d, p, R);
        for (int n = 0; n <= p; n++)
            for (int m = 0; m <= n; m++)
                M[tri(n, m)] += q[j] * conj(signed_view(R, n, m));
    }
    free(R);
}

/*
 * M2M: shift a multipole expansion about c_child to c_parent and add it:
 * M'_n^m += sum_{k<=n} sum_l conj(Upsilon_k^l(c_child - c_parent)) M_{n-k}^{m-l}.
 */
void orc_m2m(const cplx *Mc, const double cc[3], const double cp[3], int p, cplx *Mp)
{
    cplx *R = malloc(sizeof(cplx) * orc_ncoef(p));
    double d[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
    orc_regular(d, p, R);
    for (int n = 0; n <= p; n++)
        for (int m = 0; m <= n; m++) {
            cplx s = 0.0;
            for (int k = 0; k <= n; k++)
                for (int l = -k; l <= k; l++)
                    s += conj(signed_view(R, k, l)) * coef(Mc, n - k, m - l);
            Mp[tri(n, m)] += s;
        }
    free(R);
}

/*
 * M2L in its basic O(p^4) form: for a multipole expansion about c_s and a
 * local expansion about c_t,
 *   L_k^l += (-1)^k sum_{n<=p} sum_m M_n^m Theta_{n+k}^{m+l}(c_t - c_s),
 * truncated at k <= p (square truncation).
 */
void orc_m2l(const cplx *Ms, const double cs[3], const double ct[3], int p, cplx *Lt)
{
    cplx *T = malloc(sizeof(cplx) * orc_ncoef(2 * p));
    double d[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
    orc_irregular(d, 2 * p, T);
    for (int k = 0; k <= p; k++)
        for (int l = 0; l <= k; l++) {
            cplx s = 0.0;
            for (int n = 0; n <= p; n++)
                for (int m = -n; m <= n; m++)
                    s += coef(Ms, n, m) * signed_view(T, n + k, m + l);
            Lt[tri(k, l)] += (k & 1) ? -s : s;
        }
    free(T);
}

/*
 * L2L: re-centre a local expansion from c_parent to c_child and add it:
 * L'_j^i += sum_{k>=j} sum_l L_k^l conj(Upsilon_{k-j}^{l-i}(c_child - c_parent)).
 */
void orc_l2l(const cplx *Lp, const double cp[3], const double cc[3], int p, cplx *Lc)
{
    cplx *R = malloc(sizeof(cplx) * orc_ncoef(p));
    double d[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
    orc_regular(d, p, R);
    for (int j = 0; j <= p; j++)
        for (int i = 0; i <= j; i++) {
            cplx s = 0.0;
            for (int k = j; k <= p; k++)
                for (int l = -k; l <= k; l++)
                    s += coef(Lp, k, l) * conj(signed_view(R, k - j, l - i));
            Lc[tri(j, i)] += s;
        }
    free(R);
}

/*
 * L2P: phi(x) = sum_{k,l} L_k^l conj(Upsilon_k^l(x - c)); the field E = -grad phi
 * comes from the degree-1 coefficients of the expansion re-centred at x
 * (the L2L formula with d = x - c): with L1_i = sum_{k>=1,l} L_k^l
 * conj(Upsilon_{k-1}^{l-i}(x - c)), E = (Re L1_1, Im L1_1, -L1_0).
 */
void orc_l2p(const cplx *L, const double c[3], int p, const double x[3],
             double *phi, double E[3])
{
    cplx *R = malloc(sizeof(cplx) * orc_ncoef(p));
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    orc_regular(d, p, R);
    cplx s0 = 0.0, s10 = 0.0, s11 = 0.0;
    for (int k = 0; k <= p; k++)
        for (int l = -k; l <= k; l++) {
            cplx Lk = coef(L, k, l);
            s0 += Lk * conj(signed_view(R, k, l));
            if (k >= 1) {
                s10 += Lk * conj(signed_view(R, k - 1, l));
                s11 += Lk * conj(signed_view(R, k - 1, l - 1));
            }
        }
    *phi = creal(s0);
    E[0] = creal(s11);
    E[1] = cimag(s11);
    E[2] = -creal(s10);
    free(R);
}

/* ------------------------------------------------------------------ */
/* Exact pairwise sum, Eq. 2.1                                         */
/* ------------------------------------------------------------------ */

/* Neumaier-compensated accumulation. */
static void nsum(double *s, double *c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v))
        *c += (*s - t) + v;
    else
        *c += (v - t) + *s;
    *s = t;
}

/*
 * Direct sum at the given targets: phi_i = sum_{j != i} q_j / |x_i - x_j| and
 * E_i = sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3, sources in index order,
 * compensated summation. Pairs at zero distance are skipped.
 */
void orc_direct(int64_t n, const double *x, const double *q, int64_t nt,
                const int64_t *targets, double *phi, double *E)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
        for (int64_t j = 0; j < n; j++) {
            double dx = x[3 * i] - x[3 * j];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0)
                continue;
            double r = sqrt(r2);
            double qr3 = q[j] / (r2 * r);
            nsum(&s[0], &c[0], q[j] / r);
            nsum(&s[1], &c[1], qr3 * dx);
            nsum(&s[2], &c[2], qr3 * dy);
            nsum(&s[3], &c[3], qr3 * dz);
        }
        phi[t] = s[0] + c[0];
        if (E) {
            E[3 * t] = s[1] + c[1];
            E[3 * t + 1] = s[2] + c[2];
            E[3 * t + 2] = s[3] + c[3];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Tree (Algorithm 2, Sec. 2.1.2 with eta = 1)                          */
/* ------------------------------------------------------------------ */

typedef struct {
    double key;
    int64_t idx;
} orc_key;

static int key_cmp(const void *a, const void *b)
{
    const orc_key *u = a, *v = b;
    if (u->key < v->key) return -1;
    if (u->key > v->key) return 1;
    return (u->idx > v->idx) - (u->idx < v->idx);
}

typedef struct {
    int64_t n;
    int levels, p;
    double theta;
    double eta;         /* adaptivity parameter of Sec. 2.1.2, [0, 1] */
    int step;           /* bisections per FMM level (1 binary, 3 octree) */
    int tight;          /* 1: centre/radius from each box's points (see above) */
    double *x;          /* n x 3 canonical positions (-0.0 -> +0.0), input order */
    int64_t *perm;      /* slot -> original index, leaf order */
    int64_t *begin;     /* per box (heap order), first slot; nbox + 1 entries by level */
    int64_t *count;     /* per box, number of points */
    double *lo, *hi;    /* per box cell, 3 each */
    double *centre, *radius;
    int *axis;          /* per box, split axis (boxes above the leaves) */
    double *plane;      /* per box, split coordinate */
    /* connectivity per level: CSR over target boxes of that level */
    int64_t **wptr, **sptr;
    int32_t **wsrc, **ssrc;
    /* expansions per box (heap order) */
    cplx *M, *L;
} orc_fmm;

static int64_t nbox_of(int levels) { return ((int64_t)2 << levels) - 1; }
static int64_t gid(int l, int64_t j) { return ((int64_t)1 << l) - 1 + j; }

static void set_geometry(orc_fmm *F, int64_t g)
{
    double e[3];
    for (int a = 0; a < 3; a++) {
        e[a] = F->hi[3 * g + a] - F->lo[3 * g + a];
        F->centre[3 * g + a] = 0.5 * (F->lo[3 * g + a] + F->hi[3 * g + a]);
    }
    F->radius[g] = 0.5 * sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
    int ax = 0;
    if (e[1] > e[ax]) ax = 1;
    if (e[2] > e[ax]) ax = 2;
    F->axis[g] = ax;
}

/*
 * Build the balanced tree: levels binary median bisections of the tight
 * bounding box. Each box's point list is kept in ascending original index;
 * the left child takes the floor(n/2) smallest (coordinate, index) keys.
 */
static void orc_build_tree(orc_fmm *F, const double *root_lo, const double *root_hi)
{
    int64_t n = F->n, nb = nbox_of(F->levels);
    int64_t *lists = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *tmp = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    orc_key *keys = malloc(sizeof(orc_key) * (n > 0 ? n : 1));
    char *left = malloc(n > 0 ? n : 1);
    for (int64_t i = 0; i < n; i++)
        lists[i] = i;
    /* root cell: tight bounding box, or the given cell (a box of a larger
     * tree, whose subtree this tree then is) */
    for (int a = 0; a < 3; a++) {
        double lo = F->x[a], hi = F->x[a];
        for (int64_t i = 1; i < n; i++) {
            if (F->x[3 * i + a] < lo) lo = F->x[3 * i + a];
            if (F->x[3 * i + a] > hi) hi = F->x[3 * i + a];
        }
        F->lo[a] = root_lo ? root_lo[a] + 0.0 : lo;
        F->hi[a] = root_hi ? root_hi[a] + 0.0 : hi;
    }
    F->begin[0] = 0;
    F->count[0] = n;
    set_geometry(F, 0);
    for (int l = 0; l < F->levels; l++) {
        for (int64_t j = 0; j < ((int64_t)1 << l); j++) {
            int64_t g = gid(l, j), b = F->begin[g], nn = F->count[g];
            int ax = F->axis[g];
            int64_t k = nn / 2;
            for (int64_t t = 0; t < nn; t++) {
                keys[t].key = F->x[3 * lists[b + t] + ax];
                keys[t].idx = lists[b + t];
            }
            qsort(keys, nn, sizeof(orc_key), key_cmp);
            for (int64_t t = 0; t < nn; t++)
                left[lists[b + t]] = 0;
            for (int64_t t = 0; t < k; t++)
                left[keys[t].idx] = 1;
            double s;
            if (nn >= 2)
                s = 0.5 * (keys[k - 1].key + keys[k].key);
            else if (nn == 1)
                s = keys[0].key;
            else
                s = 0.5 * (F->lo[3 * g + ax] + F->hi[3 * g + ax]);
            if (F->eta < 1.0) {
                /* eta in [0, 1): the plane is the weighted average of the median
                 * plane and the geometric midpoint (Sec. 2.1.2); the left child
                 * takes the points strictly below it */
                double mid = 0.5 * (F->lo[3 * g + ax] + F->hi[3 * g + ax]);
                s = F->eta * s + (1.0 - F->eta) * mid;
                k = 0;
                for (int64_t t = 0; t < nn; t++) {
                    left[lists[b + t]] = F->x[3 * lists[b + t] + ax] < s;
                    k += left[lists[b + t]];
                }
            }
            F->plane[g] = s;
            /* stable partition of the ascending-index list */
            int64_t nl = 0, nr = 0;
            for (int64_t t = 0; t < nn; t++)
                if (left[lists[b + t]])
                    tmp[nl++] = lists[b + t];
            for (int64_t t = 0; t < nn; t++)
                if (!left[lists[b + t]])
                    tmp[k + nr++] = lists[b + t];
            memcpy(lists + b, tmp, sizeof(int64_t) * nn);
            int64_t cl = gid(l + 1, 2 * j), cr = gid(l + 1, 2 * j + 1);
            F->begin[cl] = b;
            F->count[cl] = k;
            F->begin[cr] = b + k;
            F->count[cr] = nn - k;
            for (int a = 0; a < 3; a++) {
                F->lo[3 * cl + a] = F->lo[3 * g + a];
                F->hi[3 * cl + a] = F->hi[3 * g + a];
                F->lo[3 * cr + a] = F->lo[3 * g + a];
                F->hi[3 * cr + a] = F->hi[3 * g + a];
            }
            F->hi[3 * cl + ax] = s;
            F->lo[3 * cr + ax] = s;
            set_geometry(F, cl);
            set_geometry(F, cr);
        }
    }
    memcpy(F->perm, lists, sizeof(int64_t) * n);
    free(lists);
    free(tmp);
    free(keys);
    free(left);
}

/*
 * Tight box geometry: the bounding box of a box's points, its midpoint as
 * the expansion centre and its half diagonal as the radius, floored at 2^-10
 * of the cell radius. Min and max are exact, so the result does not depend
 * on the order in which the points are visited.
 */
static void orc_tight_geometry(orc_fmm *F)
{
    int64_t nb = nbox_of(F->levels);
    for (int64_t g = 0; g < nb; g++) {
        double floor_r = ldexp(F->radius[g], -10);
        int64_t b = F->begin[g], nn = F->count[g];
        if (nn == 0) {
            F->radius[g] = floor_r;
            continue;
        }
        double lo[3], hi[3], e[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = hi[a] = F->x[3 * F->perm[b] + a];
            for (int64_t t = 1; t < nn; t++) {
                double v = F->x[3 * F->perm[b + t] + a];
                if (v < lo[a]) lo[a] = v;
                if (v > hi[a]) hi[a] = v;
            }
            e[a] = hi[a] - lo[a];
            F->centre[3 * g + a] = 0.5 * (lo[a] + hi[a]);
        }
        double r = 0.5 * sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
        F->radius[g] = r > floor_r ? r : floor_r;
    }
}

/*
 * One median bisection of a single box (Sec. 2.1.2, eta = 1), for checking
 * sampled boxes of a large tree one at a time: x holds the box's nn points
 * (nn x 3) in ascending original index, [lo, hi] its cell. The split axis is
 * the first longest cell extent; left[t] = 1 for the floor(nn/2) smallest
 * (coordinate, position) keys; returns the axis and writes the plane.
 */
int orc_bisect_box(int64_t nn, const double *x, const double lo[3], const double hi[3],
                   char *left, double *plane)
{
    double e[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    int ax = 0;
    if (e[1] > e[ax]) ax = 1;
    if (e[2] > e[ax]) ax = 2;
    orc_key *keys = malloc(sizeof(orc_key) * (nn > 0 ? nn : 1));
    for (int64_t t = 0; t < nn; t++) {
        keys[t].key = x[3 * t + ax] + 0.0;
        keys[t].idx = t;
        left[t] = 0;
    }
    qsort(keys, nn, sizeof(orc_key), key_cmp);
    int64_t k = nn / 2;
    for (int64_t t = 0; t < k; t++)
        left[keys[t].idx] = 1;
    if (nn >= 2)
        *plane = 0.5 * (keys[k - 1].key + keys[k].key);
    else if (nn == 1)
        *plane = keys[0].key;
    else
        *plane = 0.5 * (lo[ax] + hi[ax]);
    free(keys);
    return ax;
}

/* ------------------------------------------------------------------ */
/* Connectivity (Eq. 2.2 and the inheritance rule of Sec. 2.1.1)        */
/* ------------------------------------------------------------------ */

/* theta-criterion: boxes are weakly connected iff R + theta*r <= theta*d. */
int orc_theta_weak(double theta, const double ca[3], double ra, const double cb[3], double rb)
{
    double dx = ca[0] - cb[0], dy = ca[1] - cb[1], dz = ca[2] - cb[2];
    double d = sqrt((dx * dx + dy * dy) + dz * dz);
    double R = ra > rb ? ra : rb;
    double r = ra > rb ? rb : ra;
    return theta > 0.0 && d > 0.0 && R + theta * r <= theta * d;
}

/*
 * Level by level from the root's self-connection: the children of every
 * strongly connected pair are tested; weak pairs are stored for M2L at that
 * level, strong pairs are refined further and, at the leaves, form the P2P
 * list. Both orientations of every pair are stored; sources ascending.
 */
static void orc_build_lists(orc_fmm *F)
{
    int B = F->levels, st = F->step;
    int64_t C = (int64_t)1 << st; /* children per box per FMM level */
    F->wptr = calloc(B + 1, sizeof(int64_t *));
    F->sptr = calloc(B + 1, sizeof(int64_t *));
    F->wsrc = calloc(B + 1, sizeof(int32_t *));
    F->ssrc = calloc(B + 1, sizeof(int32_t *));
    F->wptr[0] = calloc(2, sizeof(int64_t));
    F->wsrc[0] = malloc(sizeof(int32_t));
    F->sptr[0] = calloc(2, sizeof(int64_t));
    F->ssrc[0] = malloc(sizeof(int32_t));
    F->sptr[0][1] = 1;
    F->ssrc[0][0] = 0;
    for (int l = 1; l <= B; l++) {
        int64_t nt = (int64_t)1 << l;
        int64_t *pw = calloc(nt + 1, sizeof(int64_t)), *ps = calloc(nt + 1, sizeof(int64_t));
        if (l % st != 0) {
            /* a bisection level inside an FMM level: no connectivity */
            F->wptr[l] = pw;
            F->sptr[l] = ps;
            F->wsrc[l] = malloc(sizeof(int32_t));
            F->ssrc[l] = malloc(sizeof(int32_t));
            continue;
        }
        int lp = l - st; /* parent FMM level */
        /* count */
        for (int64_t t = 0; t < nt; t++) {
            int64_t T = t / C, gt = gid(l, t);
            for (int64_t e = F->sptr[lp][T]; e < F->sptr[lp][T + 1]; e++) {
                int64_t S = F->ssrc[lp][e];
                for (int64_t c = 0; c < C; c++) {
                    int64_t gs = gid(l, C * S + c);
                    if (orc_theta_weak(F->theta, F->centre + 3 * gt, F->radius[gt],
                                       F->centre + 3 * gs, F->radius[gs]))
                        pw[t + 1]++;
                    else
                        ps[t + 1]++;
                }
            }
        }
        for (int64_t t = 0; t < nt; t++) {
            pw[t + 1] += pw[t];
            ps[t + 1] += ps[t];
        }
        int32_t *sw = malloc(sizeof(int32_t) * (pw[nt] + 1));
        int32_t *ss = malloc(sizeof(int32_t) * (ps[nt] + 1));
        for (int64_t t = 0; t < nt; t++) {
            int64_t T = t / C, gt = gid(l, t), iw = pw[t], is = ps[t];
            for (int64_t e = F->sptr[lp][T]; e < F->sptr[lp][T + 1]; e++) {
                int64_t S = F->ssrc[lp][e];
                for (int64_t c = 0; c < C; c++) {
                    int64_t s = C * S + c, gs = gid(l, s);
                    if (orc_theta_weak(F->theta, F->centre + 3 * gt, F->radius[gt],
                                       F->centre + 3 * gs, F->radius[gs]))
                        sw[iw++] = (int32_t)s;
                    else
                        ss[is++] = (int32_t)s;
                }
            }
        }
        F->wptr[l] = pw;
        F->sptr[l] = ps;
        F->wsrc[l] = sw;
        F->ssrc[l] = ss;
    }
}

/* ------------------------------------------------------------------ */
/* Public handle                                                        */
/* ------------------------------------------------------------------ */

orc_fmm *orc_build(int64_t n, const double *x, int levels, int p, double theta, double eta,
                   int step, int tight, const double *root_lo, const double *root_hi)
{
    if (step < 1 || levels % step != 0)
        return NULL;
    orc_fmm *F = calloc(1, sizeof(orc_fmm));
    int64_t nb = nbox_of(levels);
    F->eta = eta;
    F->step = step;
    F->tight = tight;
    F->n = n;
    F->levels = levels;
    F->p = p;
    F->theta = theta;
    F->x = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    for (int64_t i = 0; i < 3 * n; i++)
        F->x[i] = x[i] + 0.0; /* -0.0 -> +0.0 */
    F->perm = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    F->begin = calloc(nb, sizeof(int64_t));
    F->count = calloc(nb, sizeof(int64_t));
    F->lo = calloc(3 * nb, sizeof(double));
    F->hi = calloc(3 * nb, sizeof(double));
    F->centre = calloc(3 * nb, sizeof(double));
    F->radius = calloc(nb, sizeof(double));
    F->axis = calloc(nb, sizeof(int));
    F->plane = calloc(nb, sizeof(double));
    F->M = calloc(nb * orc_ncoef(p), sizeof(cplx));
    F->L = calloc(nb * orc_ncoef(p), sizeof(cplx));
    orc_build_tree(F, root_lo, root_hi);
    if (F->tight)
        orc_tight_geometry(F);
    orc_build_lists(F);
    return F;
}

void orc_free(orc_fmm *F)
{
    if (!F) return;
    for (int l = 0; l <= F->levels; l++) {
        free(F->wptr[l]);
        free(F->sptr[l]);
        free(F->wsrc[l]);
        free(F->ssrc[l]);
    }
    free(F->wptr); free(F->sptr); free(F->wsrc); free(F->ssrc);
    free(F->x); free(F->perm); free(F->begin); free(F->count);
    free(F->lo); free(F->hi); free(F->centre); free(F->radius);
    free(F->axis); free(F->plane); free(F->M); free(F->L);
    free(F);
}

int64_t orc_nbox(const orc_fmm *F) { return nbox_of(F->levels); }

void orc_get_tree(const orc_fmm *F, int64_t *perm, int64_t *begin, int64_t *count,
                  double *lo, double *hi, double *centre, double *radius,
                  int32_t *axis, double *plane)
{
    int64_t nb = nbox_of(F->levels);
    memcpy(perm, F->perm, sizeof(int64_t) * F->n);
    memcpy(begin, F->begin, sizeof(int64_t) * nb);
    memcpy(count, F->count, sizeof(int64_t) * nb);
    memcpy(lo, F->lo, sizeof(double) * 3 * nb);
    memcpy(hi, F->hi, sizeof(double) * 3 * nb);
    memcpy(centre, F->centre, sizeof(double) * 3 * nb);
    memcpy(radius, F->radius, sizeof(double) * nb);
    for (int64_t g = 0; g < nb; g++)
        axis[g] = F->axis[g];
    memcpy(plane, F->plane, sizeof(double) * nb);
}

/* kind 0 = weak (M2L) list, kind 1 = strong list (P2P at the leaf level). */
int64_t orc_list_size(const orc_fmm *F, int level, int kind)
{
    int64_t nt = (int64_t)1 << level;
    return kind == 0 ? F->wptr[level][nt] : F->sptr[level][nt];
}

void orc_get_list(const orc_fmm *F, int level, int kind, int64_t *ptr, int32_t *src)
{
    int64_t nt = (int64_t)1 << level;
    const int64_t *pp = kind == 0 ? F->wptr[level] : F->sptr[level];
    const int32_t *ss = kind == 0 ? F->wsrc[level] : F->ssrc[level];
    memcpy(ptr, pp, sizeof(int64_t) * (nt + 1));
    memcpy(src, ss, sizeof(int32_t) * pp[nt]);
}

/*
 * The FMM evaluation in the order of Algorithm 1: P2M at the leaves, M2M
 * upward, M2L at every level, L2L downward, then L2P and P2P at the leaves.
 * Outputs are in input order.
 */
void orc_eval(orc_fmm *F, const double *q, double *phi, double *E)
{
    int B = F->levels, p = F->p, nc = orc_ncoef(p);
    int64_t nb = nbox_of(B), nleaf = (int64_t)1 << B;
    memset(F->M, 0, sizeof(cplx) * nb * nc);
    memset(F->L, 0, sizeof(cplx) * nb * nc);
    double *xl = malloc(sizeof(double) * 3 * (F->n > 0 ? F->n : 1));
    double *ql = malloc(sizeof(double) * (F->n > 0 ? F->n : 1));
    for (int64_t s = 0; s < F->n; s++) {
        int64_t i = F->perm[s];
        xl[3 * s] = F->x[3 * i];
        xl[3 * s + 1] = F->x[3 * i + 1];
        xl[3 * s + 2] = F->x[3 * i + 2];
        ql[s] = q[i];
    }
    /* P2M */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < nleaf; j++) {
        int64_t g = gid(B, j);
        orc_p2m(F->count[g], xl + 3 * F->begin[g], ql + F->begin[g],
                F->centre + 3 * g, p, F->M + g * nc);
    }
    /* M2M, leaves to root, over FMM levels (each box from its C children) */
    int st = F->step;
    int64_t C = (int64_t)1 << st;
    for (int l = B; l >= st; l -= st)
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t j = 0; j < ((int64_t)1 << (l - st)); j++) {
            int64_t gp = gid(l - st, j);
            for (int64_t c = 0; c < C; c++) {
                int64_t gc = gid(l, C * j + c);
                orc_m2m(F->M + gc * nc, F->centre + 3 * gc, F->centre + 3 * gp, p,
                        F->M + gp * nc);
            }
        }
    /* M2L at every level */
    for (int l = 1; l <= B; l++)
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t t = 0; t < ((int64_t)1 << l); t++) {
            int64_t gt = gid(l, t);
            for (int64_t e = F->wptr[l][t]; e < F->wptr[l][t + 1]; e++) {
                int64_t gs = gid(l, F->wsrc[l][e]);
                orc_m2l(F->M + gs * nc, F->centre + 3 * gs, F->centre + 3 * gt, p,
                        F->L + gt * nc);
            }
        }
    /* L2L, root to leaves, over FMM levels */
    for (int l = st; l <= B; l += st)
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t j = 0; j < ((int64_t)1 << l); j++) {
            int64_t gc = gid(l, j), gp = gid(l - st, j / C);
            orc_l2l(F->L + gp * nc, F->centre + 3 * gp, F->centre + 3 * gc, p,
                    F->L + gc * nc);
        }
    /* L2P and P2P at the leaves */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nleaf; t++) {
        int64_t gt = gid(B, t);
        for (int64_t a = F->begin[gt]; a < F->begin[gt] + F->count[gt]; a++) {
            double f, e[3];
            orc_l2p(F->L + gt * nc, F->centre + 3 * gt, p, xl + 3 * a, &f, e);
            for (int64_t s = F->sptr[B][t]; s < F->sptr[B][t + 1]; s++) {
                int64_t gs = gid(B, F->ssrc[B][s]);
                for (int64_t b = F->begin[gs]; b < F->begin[gs] + F->count[gs]; b++) {
                    double dx = xl[3 * a] - xl[3 * b];
                    double dy = xl[3 * a + 1] - xl[3 * b + 1];
                    double dz = xl[3 * a + 2] - xl[3 * b + 2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0)
                        continue;
                    double r = sqrt(r2);
                    double qr3 = ql[b] / (r2 * r);
                    f += ql[b] / r;
                    e[0] += qr3 * dx;
                    e[1] += qr3 * dy;
                    e[2] += qr3 * dz;
                }
            }
            int64_t i = F->perm[a];
            phi[i] = f;
            if (E) {
                E[3 * i] = e[0];
                E[3 * i + 1] = e[1];
                E[3 * i + 2] = e[2];
            }
        }
    }
    free(xl);
    free(ql);
}

/* Copy of the multipole (which == 0) or local (which == 1) coefficients of
 * every box, heap order, as (re, im) pairs. */
void orc_get_expansions(const orc_fmm *F, int which, double *out)
{
    int64_t tot = nbox_of(F->levels) * orc_ncoef(F->p);
    const cplx *C = which == 0 ? F->M : F->L;
    for (int64_t i = 0; i < tot; i++) {
        out[2 * i] = creal(C[i]);
        out[2 * i + 1] = cimag(C[i]);
    }
}

/* Number of worker threads the oracle's parallel loops use. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
