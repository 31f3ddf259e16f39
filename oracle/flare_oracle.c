/*
 * FP64 CPU oracle of the FLARE mapped-sparse-GP energy / force / uncertainty
 * path (paper Sec. V-B, Eq. 1 and Eq. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with
 * the CUDA implementation.
 *
 * It is the plain definition written out, slow and in double precision:
 *
 *   neighbours    all (j, image) with |r_j + S.cell - r_i| < r_c   (Sec. V-B,
 *                 "local atomic environment ... within a cutoff radius")
 *   basis         phi_{n,l,m}(r) = T_n(2|r|/r_cut - 1) (r_cut - |r|)^2 Y_lm(r/|r|)
 *                 (radial functions and spherical harmonics of the ACE basis,
 *                 Sec. V-B; the radial form and cutoff are this
 *                 implementation's reading because the paper does not print them)
 *   A             A_{i,(s,n),l,m} = sum over neighbours j of species s of phi
 *   B2            B_{(a,b),l} = sum_m A_{a,l,m} A_{b,l,m},  a <= b
 *   descriptor    d = B / ||B||  (Sec. V-B, normalized ACE-B2)
 *   energy        E_i = d^T beta_{s_i} d              (Eq. 1, mapped form)
 *   variance      V_i = d^T Sigma_{s_i} d             (Eq. 2, mapped form)
 *   forces        F_k = -dE/dr_k, formed the un-reordered way: the dense
 *                 Jacobian of d_i with respect to every neighbour vector is
 *                 built and contracted with dE_i/dd_i.  The GPU path uses the
 *                 reordered summation of Sec. V-B ("Acceleration of force
 *                 predictions"), so agreement checks that reordering.
 *
 * Derivatives of the basis are taken by the complex-step method
 * (Squire and Trapp, SIAM Review 40, 1998): for a function analytic in its
 * argument, d f / d x = Im f(x + i h) / h exactly up to rounding for tiny h.
 * This is independent of the analytic gradients used on the GPU.
 *
 * Descriptor component order: index = tri(a, b) * (L + 1) + l with channels
 * a = s * N + n, a <= b, tri() row-major over the upper triangle.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_LMAX 3
#define ORC_NLM ((ORC_LMAX + 1) * (ORC_LMAX + 1))

/* ------------------------------------------------------------------ */
/* Real orthonormal spherical harmonics, l <= 3, of a (complex) unit    */
/* vector u.  Index l*l + (m + l), m = -l..l.  The normalisation makes  */
/* sum_m Y_lm^2 = (2l + 1) / (4 pi) on the real unit sphere.            */
/* ------------------------------------------------------------------ */
static void orc_ylm(cplx x, cplx y, cplx z, int l_max, cplx *Y)
{
    const double pi = M_PI;
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (l_max < 1) return;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = k1 * y;
    Y[2] = k1 * z;
    Y[3] = k1 * x;
    if (l_max < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k20 = 0.25 * sqrt(5.0 / pi);
    const double k22 = 0.25 * sqrt(15.0 / pi);
    Y[4] = k2a * x * y;
    Y[5] = k2a * y * z;
    Y[6] = k20 * (3.0 * z * z - 1.0);
    Y[7] = k2a * x * z;
    Y[8] = k22 * (x * x - y * y);
    if (l_max < 3) return;
    const double k33 = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k32 = 0.5 * sqrt(105.0 / pi);
    const double k31 = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k30 = 0.25 * sqrt(7.0 / pi);
    const double k32b = 0.25 * sqrt(105.0 / pi);
    Y[9] = k33 * y * (3.0 * x * x - y * y);
    Y[10] = k32 * x * y * z;
    Y[11] = k31 * y * (5.0 * z * z - 1.0);
    Y[12] = k30 * (5.0 * z * z * z - 3.0 * z);
    Y[13] = k31 * x * (5.0 * z * z - 1.0);
    Y[14] = k32b * z * (x * x - y * y);
    Y[15] = k33 * x * (x * x - 3.0 * y * y);
}

/* phi[n * nlm + lm] for the (complex) neighbour vector r; zero beyond r_cut. */
static void orc_basis_c(const cplx r[3], int n_max, int l_max, double r_cut, cplx *phi)
{
    const int nlm = (l_max + 1) * (l_max + 1);
    cplx rr = csqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(creal(rr) < r_cut)) {
        for (int k = 0; k < n_max * nlm; ++k) phi[k] = 0.0;
        return;
    }
    cplx Y[ORC_NLM];
    orc_ylm(r[0] / rr, r[1] / rr, r[2] / rr, l_max, Y);
    cplx x = 2.0 * rr / r_cut - 1.0;
    cplx fc = (r_cut - rr) * (r_cut - rr);
    cplx t_prev = 1.0, t_cur = x;      /* Chebyshev T_0, T_1 */
    for (int n = 0; n < n_max; ++n) {
        cplx T;
        if (n == 0) T = 1.0;
        else if (n == 1) T = x;
        else {
            T = 2.0 * x * t_cur - t_prev;
            t_prev = t_cur;
            t_cur = T;
        }
        for (int lm = 0; lm < nlm; ++lm) phi[n * nlm + lm] = T * fc * Y[lm];
    }
}

/* Real basis values and their complex-step gradients with respect to r. */
static void orc_basis_grad(const double r[3], int n_max, int l_max, double r_cut,
                           double *phi, double *dphi /* [n*nlm][3] */)
{
    const int nb = n_max * (l_max + 1) * (l_max + 1);
    const double h = 1e-30;
    cplx rc[3] = {r[0], r[1], r[2]};
    cplx tmp[8 * ORC_NLM * 4];
    cplx *buf = tmp;
    cplx *heap = NULL;
    if (nb > 8 * ORC_NLM * 4) { heap = malloc(sizeof(cplx) * nb); buf = heap; }
    orc_basis_c(rc, n_max, l_max, r_cut, buf);
    for (int k = 0; k < nb; ++k) phi[k] = creal(buf[k]);
    for (int c = 0; c < 3; ++c) {
        cplx rp[3] = {r[0], r[1], r[2]};
        rp[c] += I * h;
        orc_basis_c(rp, n_max, l_max, r_cut, buf);
        for (int k = 0; k < nb; ++k) dphi[3 * k + c] = cimag(buf[k]) / h;
    }
    free(heap);
}

/* ------------------------------------------------------------------ */
/* Cell geometry                                                        */
/* ------------------------------------------------------------------ */
static void orc_inverse3(const double *m, double *inv)
{
    double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                 m[2] * (m[3] * m[7] - m[4] * m[6]);
    inv[0] = (m[4] * m[8] - m[5] * m[7]) / det;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    inv[3] = (m[5] * m[6] - m[3] * m[8]) / det;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    inv[6] = (m[3] * m[7] - m[4] * m[6]) / det;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

/* Perpendicular width of the cell along lattice direction d:
   volume / |a_e x a_f|. */
static double orc_width(const double *cell, int d)
{
    const double *a = cell, *b = cell + 3, *c = cell + 6;
    double vol = fabs(a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                      a[2] * (b[0] * c[1] - b[1] * c[0]));
    const double *e = cell + 3 * ((d + 1) % 3), *f = cell + 3 * ((d + 2) % 3);
    double x = e[1] * f[2] - e[2] * f[1], y = e[2] * f[0] - e[0] * f[2], z = e[0] * f[1] - e[1] * f[0];
    return vol / sqrt(x * x + y * y + z * z);
}

static void orc_image_vec(const double *cell, int sx, int sy, int sz, double *t)
{
    for (int c = 0; c < 3; ++c) t[c] = sx * cell[c] + sy * cell[3 + c] + sz * cell[6 + c];
}

typedef struct { int i, j, s[3]; } orc_pair;

static int orc_pair_cmp(const void *pa, const void *pb)
{
    const orc_pair *a = pa, *b = pb;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    for (int c = 0; c < 3; ++c)
        if (a->s[c] != b->s[c]) return a->s[c] < b->s[c] ? -1 : 1;
    return 0;
}

/*
 * Brute-force neighbour search: every ordered pair (i, j) and every lattice
 * image S with |S_d| <= ceil(r_c / width_d) + 1 along periodic directions,
 * kept when |r_j + S.cell - r_i|^2 < r_c^2 and (j, S) != (i, 0).
 * Writes up to `cap` pairs as [i, j, sx, sy, sz] sorted by (i, j, S) and
 * returns the total count (call again with a larger cap if it exceeds cap).
 */
long orc_neighbors_brute(int n, const double *pos, const double *cell, const int *pbc,
                         double rc, long cap, int *out)
{
    int K[3];
    for (int d = 0; d < 3; ++d) K[d] = pbc[d] ? (int)ceil(rc / orc_width(cell, d)) + 1 : 0;
    long count = 0;
    orc_pair *buf = malloc(sizeof(orc_pair) * (cap > 0 ? cap : 1));
    const double rc2 = rc * rc;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int sx = -K[0]; sx <= K[0]; ++sx)
                for (int sy = -K[1]; sy <= K[1]; ++sy)
                    for (int sz = -K[2]; sz <= K[2]; ++sz) {
                        if (i == j && sx == 0 && sy == 0 && sz == 0) continue;
                        double t[3];
                        orc_image_vec(cell, sx, sy, sz, t);
                        double d2 = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            double dc = pos[3 * j + c] + t[c] - pos[3 * i + c];
                            d2 += dc * dc;
                        }
                        if (d2 < rc2) {
                            if (count < cap) {
                                orc_pair p = {i, j, {sx, sy, sz}};
                                buf[count] = p;
                            }
                            ++count;
                        }
                    }
    long m = count < cap ? count : cap;
    qsort(buf, m, sizeof(orc_pair), orc_pair_cmp);
    for (long k = 0; k < m; ++k) {
        out[5 * k] = buf[k].i;
        out[5 * k + 1] = buf[k].j;
        for (int c = 0; c < 3; ++c) out[5 * k + 2 + c] = buf[k].s[c];
    }
    free(buf);
    return count;
}

/*
 * Cell-list neighbour search for a subset of centre atoms (all atoms when
 * centers == NULL).  Atoms are binned by fractional coordinate (wrapped
 * along periodic directions, positions must already lie in the cell there);
 * every bin holds a slab of width >= r_c, and all images of all bins within
 * reach are visited, so the result equals the brute-force set.  Same output
 * format and order as orc_neighbors_brute.
 */
long orc_neighbors_cells(int n, const double *pos, const double *cell, const int *pbc,
                         double rc, int n_centers, const int *centers, long cap, int *out)
{
    double inv[9];
    orc_inverse3(cell, inv);
    double *frac = malloc(sizeof(double) * 3 * (size_t)n);
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) { lo[d] = 1e300; hi[d] = -1e300; }
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            /* fractional coordinate d = sum_c pos_c * inv[c][d] (pos = frac . cell) */
            double f = pos[3 * i] * inv[d] + pos[3 * i + 1] * inv[3 + d] + pos[3 * i + 2] * inv[6 + d];
            frac[3 * i + d] = f;
            if (f < lo[d]) lo[d] = f;
            if (f > hi[d]) hi[d] = f;
        }
    int nb[3], R[3];
    double flo[3], fspan[3];
    for (int d = 0; d < 3; ++d) {
        double w = orc_width(cell, d);
        if (pbc[d]) { flo[d] = 0.0; fspan[d] = 1.0; }
        else { flo[d] = lo[d]; fspan[d] = (hi[d] - lo[d]) > 0 ? (hi[d] - lo[d]) * (1 + 1e-12) : 1e-9; }
        double extent = fspan[d] * w;          /* perpendicular extent in A */
        nb[d] = (int)floor(extent / (rc * 1.001));
        if (nb[d] < 1) nb[d] = 1;
        /* bins to visit on each side so that r_c is covered */
        R[d] = (int)ceil(rc / (extent / nb[d]) * 1.000001);
        if (!pbc[d] && R[d] > nb[d]) R[d] = nb[d];
    }
    long nbins = (long)nb[0] * nb[1] * nb[2];
    int *bin_of = malloc(sizeof(int) * (size_t)n);
    long *start = calloc(nbins + 1, sizeof(long));
    for (int i = 0; i < n; ++i) {
        int b[3];
        for (int d = 0; d < 3; ++d) {
            int k = (int)floor((frac[3 * i + d] - flo[d]) / fspan[d] * nb[d]);
            if (k < 0) k = 0;
            if (k >= nb[d]) k = nb[d] - 1;
            b[d] = k;
        }
        bin_of[i] = (b[0] * nb[1] + b[1]) * nb[2] + b[2];
        start[bin_of[i] + 1]++;
    }
    for (long b = 0; b < nbins; ++b) start[b + 1] += start[b];
    long *fill = malloc(sizeof(long) * nbins);
    memcpy(fill, start, sizeof(long) * nbins);
    int *members = malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) members[fill[bin_of[i]]++] = i;   /* ascending i within bins */

    const double rc2 = rc * rc;
    long count = 0;
    int ncent = centers ? n_centers : n;
    orc_pair *buf = malloc(sizeof(orc_pair) * (cap > 0 ? cap : 1));
    orc_pair *row = NULL;
    long row_cap = 0;
    for (int c_ix = 0; c_ix < ncent; ++c_ix) {
        int i = centers ? centers[c_ix] : c_ix;
        int bi[3] = {bin_of[i] / (nb[1] * nb[2]), (bin_of[i] / nb[2]) % nb[1], bin_of[i] % nb[2]};
        long row_n = 0;
        for (int dx = -R[0]; dx <= R[0]; ++dx)
            for (int dy = -R[1]; dy <= R[1]; ++dy)
                for (int dz = -R[2]; dz <= R[2]; ++dz) {
                    int d3[3] = {dx, dy, dz}, bj[3], s[3];
                    int skip = 0;
                    for (int d = 0; d < 3; ++d) {
                        int k = bi[d] + d3[d];
                        if (pbc[d]) {
                            int q = (int)floor((double)k / nb[d]);
                            s[d] = q;
                            bj[d] = k - q * nb[d];
                        } else {
                            if (k < 0 || k >= nb[d]) skip = 1;
                            s[d] = 0;
                            bj[d] = k;
                        }
                    }
                    if (skip) continue;
                    long b = ((long)bj[0] * nb[1] + bj[1]) * nb[2] + bj[2];
                    double t[3];
                    orc_image_vec(cell, s[0], s[1], s[2], t);
                    for (long q = start[b]; q < start[b + 1]; ++q) {
                        int j = members[q];
                        if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
                        double d2 = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            double dc = pos[3 * j + c] + t[c] - pos[3 * i + c];
                            d2 += dc * dc;
                        }
                        if (d2 < rc2) {
                            if (row_n == row_cap) {
                                row_cap = row_cap ? 2 * row_cap : 256;
                                row = realloc(row, sizeof(orc_pair) * row_cap);
                            }
                            orc_pair p = {i, j, {s[0], s[1], s[2]}};
                            row[row_n++] = p;
                        }
                    }
                }
        qsort(row, row_n, sizeof(orc_pair), orc_pair_cmp);
        for (long k = 0; k < row_n; ++k) {
            if (count < cap) buf[count] = row[k];
            ++count;
        }
    }
    long m = count < cap ? count : cap;
    for (long k = 0; k < m; ++k) {
        out[5 * k] = buf[k].i;
        out[5 * k + 1] = buf[k].j;
        for (int c = 0; c < 3; ++c) out[5 * k + 2 + c] = buf[k].s[c];
    }
    free(row); free(buf); free(members); free(fill); free(start); free(bin_of); free(frac);
    return count;
}

/* ------------------------------------------------------------------ */
/* Per-centre evaluation                                                */
/* ------------------------------------------------------------------ */
static inline int orc_tri(int a, int b, int C)
{
    /* row-major index of (a, b), a <= b, in the upper triangle of a C x C matrix */
    return a * C - a * (a - 1) / 2 + (b - a);
}

/*
 * Evaluate every centre i with flag[i] != 0 (all centres when flag == NULL).
 * `pairs` = [n_pairs][5] rows (i, j, sx, sy, sz) sorted by i; for every
 * evaluated centre its list must be complete for r < r_cut (pairs farther
 * than r_cut are allowed and ignored).
 *
 * Outputs (any may be NULL):
 *   A_out   [n][S*N*(L+1)^2]     B_out/dhat_out [n][d]   norm_out [n]
 *   E_out, V_out [n]             fpair [n_pairs][3] = dE_i/dr_ij for pair (i, j, S)
 *   rij_out [n_pairs][3] = r_j + S.cell - r_i
 * beta, sigma: [S][d][d] row-major.
 */
int orc_evaluate(int n_species, int n_max, int l_max, double r_cut,
                 int n, const double *pos, const int *species, const double *cell,
                 long n_pairs, const int *pairs, const double *beta, const double *sigma,
                 const int *flag, int n_threads,
                 double *A_out, double *B_out, double *dhat_out, double *norm_out,
                 double *E_out, double *V_out, double *fpair, double *rij_out)
{
    if (l_max > ORC_LMAX || l_max < 0 || n_max < 1 || n_species < 1) return 1;
    const int nlm = (l_max + 1) * (l_max + 1);
    const int L1 = l_max + 1;
    const int C = n_species * n_max;
    const int d = C * (C + 1) / 2 * L1;
    const int nA = C * nlm;
    const int nb = n_max * nlm;

    long *row_start = malloc(sizeof(long) * ((size_t)n + 1));
    for (int i = 0; i <= n; ++i) row_start[i] = 0;
    for (long p = 0; p < n_pairs; ++p) row_start[pairs[5 * p] + 1]++;
    for (int i = 0; i < n; ++i) row_start[i + 1] += row_start[i];

    if (rij_out || fpair)
        for (long p = 0; p < n_pairs; ++p) {
            const int *q = pairs + 5 * p;
            double t[3];
            orc_image_vec(cell, q[2], q[3], q[4], t);
            for (int c = 0; c < 3; ++c) {
                double v = pos[3 * q[1] + c] + t[c] - pos[3 * q[0] + c];
                if (rij_out) rij_out[3 * p + c] = v;
                if (fpair) fpair[3 * p + c] = 0.0;
            }
        }

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
    int status = 0;
#pragma omp parallel
    {
        double *A = malloc(sizeof(double) * nA);
        double *B = malloc(sizeof(double) * d);
        double *dh = malloc(sizeof(double) * d);
        double *u = malloc(sizeof(double) * d);
        double *gE = malloc(sizeof(double) * d);
        double *JB = malloc(sizeof(double) * 3 * d);
        double *dA = malloc(sizeof(double) * 3 * nA);
        long cap = 64;
        double *phi = malloc(sizeof(double) * cap * nb);
        double *dphi = malloc(sizeof(double) * cap * nb * 3);
        double *rv = malloc(sizeof(double) * cap * 3);
        int *sp = malloc(sizeof(int) * cap);
        long *pid = malloc(sizeof(long) * cap);
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            if (flag && !flag[i]) continue;
            /* neighbours of i within r_cut */
            long m = 0;
            for (long p = row_start[i]; p < row_start[i + 1]; ++p) {
                const int *q = pairs + 5 * p;
                double t[3], r[3], r2 = 0.0;
                orc_image_vec(cell, q[2], q[3], q[4], t);
                for (int c = 0; c < 3; ++c) {
                    r[c] = pos[3 * q[1] + c] + t[c] - pos[3 * i + c];
                    r2 += r[c] * r[c];
                }
                if (!(r2 < r_cut * r_cut)) continue;
                if (m == cap) {
                    cap *= 2;
                    phi = realloc(phi, sizeof(double) * cap * nb);
                    dphi = realloc(dphi, sizeof(double) * cap * nb * 3);
                    rv = realloc(rv, sizeof(double) * cap * 3);
                    sp = realloc(sp, sizeof(int) * cap);
                    pid = realloc(pid, sizeof(long) * cap);
                }
                for (int c = 0; c < 3; ++c) rv[3 * m + c] = r[c];
                sp[m] = species[q[1]];
                pid[m] = p;
                orc_basis_grad(r, n_max, l_max, r_cut, phi + m * nb, dphi + m * nb * 3);
                ++m;
            }
            /* A: sum of basis values over neighbours, by neighbour species */
            for (int k = 0; k < nA; ++k) A[k] = 0.0;
            for (long p = 0; p < m; ++p) {
                int s = sp[p];
                if (s < 0 || s >= n_species) { status = 2; continue; }
                for (int k = 0; k < nb; ++k) A[s * nb + k] += phi[p * nb + k];
            }
            /* B2: contraction over m, a <= b */
            for (int a = 0; a < C; ++a)
                for (int b = a; b < C; ++b)
                    for (int l = 0; l < L1; ++l) {
                        double acc = 0.0;
                        for (int mm = 0; mm < 2 * l + 1; ++mm)
                            acc += A[a * nlm + l * l + mm] * A[b * nlm + l * l + mm];
                        B[orc_tri(a, b, C) * L1 + l] = acc;
                    }
            double nrm2 = 0.0;
            for (int k = 0; k < d; ++k) nrm2 += B[k] * B[k];
            double nrm = sqrt(nrm2);
            for (int k = 0; k < d; ++k) dh[k] = nrm > 0.0 ? B[k] / nrm : 0.0;
            int si = species[i];
            const double *bt = beta + (size_t)si * d * d;
            const double *sg = sigma + (size_t)si * d * d;
            /* Eq. 1 and Eq. 2 in their mapped quadratic forms */
            double E = 0.0, V = 0.0;
            for (int r = 0; r < d; ++r) {
                double ub = 0.0, us = 0.0;
                for (int c = 0; c < d; ++c) {
                    ub += bt[(size_t)r * d + c] * dh[c];
                    us += sg[(size_t)r * d + c] * dh[c];
                }
                u[r] = ub;
                E += dh[r] * ub;
                V += dh[r] * us;
            }
            if (A_out) memcpy(A_out + (size_t)i * nA, A, sizeof(double) * nA);
            if (B_out) memcpy(B_out + (size_t)i * d, B, sizeof(double) * d);
            if (dhat_out) memcpy(dhat_out + (size_t)i * d, dh, sizeof(double) * d);
            if (norm_out) norm_out[i] = nrm;
            if (E_out) E_out[i] = E;
            if (V_out) V_out[i] = V;
            if (!fpair || nrm == 0.0) continue;
            /* dE/dd = (beta + beta^T) d */
            for (int r = 0; r < d; ++r) {
                double acc = 0.0;
                for (int c = 0; c < d; ++c) acc += bt[(size_t)c * d + r] * dh[c];
                gE[r] = u[r] + acc;
            }
            /* Forces the un-reordered way: dense Jacobian of d wrt each neighbour vector */
            for (long p = 0; p < m; ++p) {
                int s = sp[p];
                for (int k = 0; k < 3 * nA; ++k) dA[k] = 0.0;
                for (int k = 0; k < nb; ++k)
                    for (int c = 0; c < 3; ++c) dA[3 * (s * nb + k) + c] = dphi[(p * nb + k) * 3 + c];
                /* dB_{ab,l}/dr = sum_m dA_a A_b + A_a dA_b */
                for (int a = 0; a < C; ++a)
                    for (int b = a; b < C; ++b)
                        for (int l = 0; l < L1; ++l) {
                            double acc[3] = {0, 0, 0};
                            for (int mm = 0; mm < 2 * l + 1; ++mm) {
                                int ia = a * nlm + l * l + mm, ib = b * nlm + l * l + mm;
                                for (int c = 0; c < 3; ++c)
                                    acc[c] += dA[3 * ia + c] * A[ib] + A[ia] * dA[3 * ib + c];
                            }
                            int k = orc_tri(a, b, C) * L1 + l;
                            for (int c = 0; c < 3; ++c) JB[3 * k + c] = acc[c];
                        }
                /* dd/dr = (dB - d (d . dB)) / ||B||;  f = dE/dd . dd/dr */
                double proj[3] = {0, 0, 0};
                for (int k = 0; k < d; ++k)
                    for (int c = 0; c < 3; ++c) proj[c] += dh[k] * JB[3 * k + c];
                double f[3] = {0, 0, 0};
                for (int k = 0; k < d; ++k)
                    for (int c = 0; c < 3; ++c) f[c] += gE[k] * (JB[3 * k + c] - dh[k] * proj[c]) / nrm;
                for (int c = 0; c < 3; ++c) fpair[3 * pid[p] + c] = f[c];
            }
        }
        free(A); free(B); free(dh); free(u); free(gE); free(JB); free(dA);
        free(phi); free(dphi); free(rv); free(sp); free(pid);
    }
    free(row_start);
    return status;
}

/*
 * Assemble forces and the virial from per-pair dE_i/dr_ij:
 *   F_i += f_ij, F_j -= f_ij      (r_ij = r_j + S.cell - r_i)
 *   W_ab = -sum over pairs (r_ij)_a (f_ij)_b
 * Only pairs whose centre has flag != 0 contribute (all when flag == NULL).
 */
void orc_assemble(int n, long n_pairs, const int *pairs, const double *rij, const double *fpair,
                  const int *flag, double *F, double *W)
{
    for (int k = 0; k < 3 * n; ++k) F[k] = 0.0;
    for (int k = 0; k < 9; ++k) W[k] = 0.0;
    for (long p = 0; p < n_pairs; ++p) {
        int i = pairs[5 * p], j = pairs[5 * p + 1];
        if (flag && !flag[i]) continue;
        for (int c = 0; c < 3; ++c) {
            F[3 * i + c] += fpair[3 * p + c];
            F[3 * j + c] -= fpair[3 * p + c];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) W[3 * a + b] -= rij[3 * p + a] * fpair[3 * p + b];
    }
}

/* Basis values and complex-step gradients for one vector (exposed for pins). */
void orc_basis_point(int n_max, int l_max, double r_cut, const double *r, double *phi, double *dphi)
{
    orc_basis_grad(r, n_max, l_max, r_cut, phi, dphi);
}

/* Real spherical harmonics of a real unit vector (exposed for pins). */
void orc_ylm_point(int l_max, const double *u, double *Y)
{
    cplx Yc[ORC_NLM];
    orc_ylm(u[0], u[1], u[2], l_max, Yc);
    for (int k = 0; k < (l_max + 1) * (l_max + 1); ++k) Y[k] = creal(Yc[k]);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
