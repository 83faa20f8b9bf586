/*
 * usr_oracle.c -- plain FP64 CPU oracle for u-series electrostatics
 * (Predescu et al., "The u-series: a separable decomposition for
 * electrostatics computation with improved accuracy", arXiv:1911.01377).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that
 * the GPU library is checked against.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg load it.  It shares no code, header,
 * table or constant with the GPU library; the two meet only at the seeded
 * input generators.
 *
 * Conventions: Coulomb constant 1, charges in e, lengths in Angstrom,
 * energies in e^2/Angstrom.  Orthorhombic periodic box (Sec. II).
 *
 * What is computed (double precision throughout):
 *   far function   F(r)  = sum_j a_j exp(-r^2 / (2 s_j^2))          Eqs. 19, 24, 28
 *       a_0 = c w0, s_0 = s0 sigma;  a_j = c b^-j, s_j = b^j sigma (j >= 1)
 *       c = 2 ln(b) / sqrt(2 pi sigma^2), sigma = r_c / r0           Eq. 23
 *       (Eq. 28's narrow term is read as w0 exp(-r^2/(2 s0^2 sigma^2)) / sqrt(2 pi sigma^2):
 *        the third row of Table 2 satisfies Eq. 27 only under this reading.)
 *   near function  N(r)  = 1/r - F(r) for r < r_c, 0 otherwise          Eq. 20
 *   energy E = E_near + E_far + E_self with
 *       E_near = 1/2 sum_i sum_j sum_n' q_i q_j N(|r_i - r_j + n|)      Eqs. 3, 20
 *       E_far  = 1/(2V) sum_{k != 0} Fhat(k) |S(k)|^2                   Eqs. 4, 9, F1
 *                S(k) = sum_j q_j exp(i k.r_j)
 *                Fhat(k) = sum_j a_j (2 pi s_j^2)^{3/2} exp(-s_j^2 k^2 / 2)   (App. C)
 *       E_self = -1/2 F(0) sum_i q_i^2, F(0) summed over the full series Eq. 10's self term
 *   potentials phi_i = dE/dq_i and forces F_i = -dE/dr_i.
 * The k = 0 term is dropped (Eq. 4 sums k != 0); for a non-neutral system
 * this defines E as that quadratic form of the charges.
 *
 * The far series is summed until b^-j < 1e-20 (real space) and, in k-space,
 * over every term (all j); "n_terms > 0" restricts the k-space sum to the
 * first n_terms Gaussians, the truncation studied in Sec. V / App. F.
 *
 * Also provided, as independent cross-checks for the tests:
 *   - classic Ewald (Eqs. 6-10) energies, potentials and forces;
 *   - the far part as a real-space image sum of the first N Gaussians;
 *   - the single-precision cell/pair predicate that the GPU cell list must
 *     reproduce bit for bit (documented at or_canon_cells below).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC usr_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_MAXTERMS 4096

typedef struct {
    int n;                   /* number of Gaussians kept in real space */
    double sigma;            /* sigma = r_c / r0 */
    double a[OR_MAXTERMS];   /* amplitudes */
    double s[OR_MAXTERMS];   /* widths */
} or_terms;

/* Term table of Eqs. 19/24/28 at sigma = r_c / r0 (Eq. 23). */
static void build_terms(double b, double r0, double w0, double s0, double r_c, or_terms* t)
{
    double sigma = r_c / r0;
    double c = 2.0 * log(b) / sqrt(2.0 * M_PI * sigma * sigma);
    t->sigma = sigma;
    t->a[0] = c * w0;
    t->s[0] = s0 * sigma;
    int j = 1;
    while (j < OR_MAXTERMS) {
        double bj = pow(b, (double)j);
        if (1.0 / bj < 1e-20) break;
        t->a[j] = c / bj;
        t->s[j] = sigma * bj;
        ++j;
    }
    t->n = j;
}

int or_num_terms(double b, double r0, double w0, double s0, double r_c)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    build_terms(b, r0, w0, s0, r_c, t);
    int n = t->n;
    free(t);
    return n;
}

/* Copies the first nmax (a_j, s_j) pairs; returns the number of real-space terms. */
int or_terms_table(double b, double r0, double w0, double s0, double r_c, int nmax, double* a, double* s)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    build_terms(b, r0, w0, s0, r_c, t);
    int n = t->n;
    for (int j = 0; j < nmax && j < n; ++j) { a[j] = t->a[j]; s[j] = t->s[j]; }
    free(t);
    return n;
}

static double far_F(const or_terms* t, double r)
{
    double sum = 0.0;
    for (int j = t->n - 1; j >= 0; --j)
        sum += t->a[j] * exp(-r * r / (2.0 * t->s[j] * t->s[j]));
    return sum;
}

/* dF/dr divided by r (finite at r = 0). */
static double far_dF_over_r(const or_terms* t, double r)
{
    double sum = 0.0;
    for (int j = t->n - 1; j >= 0; --j) {
        double s2 = t->s[j] * t->s[j];
        sum -= t->a[j] / s2 * exp(-r * r / (2.0 * s2));
    }
    return sum;
}

/* Fourier transform of the far function (App. C, C1 form), k > 0.  nk <= 0: all terms. */
static double far_Fhat(const or_terms* t, double k, int nk)
{
    int n = (nk > 0 && nk < t->n) ? nk : t->n;
    double sum = 0.0;
    for (int j = 0; j < n; ++j) {
        double s2 = t->s[j] * t->s[j];
        double x = 0.5 * s2 * k * k;
        if (x > 745.0) continue;
        sum += t->a[j] * pow(2.0 * M_PI * s2, 1.5) * exp(-x);
    }
    /* terms beyond the real-space table (b^-j < 1e-20) are wider than any
       box by many orders of magnitude; for k >= 2 pi / L they underflow. */
    return sum;
}

/* Evaluate F(r), F'(r)/r for an array of r (used by the tests). */
void or_far_function(double b, double r0, double w0, double s0, double r_c,
                     int n, const double* r, double* F, double* dF_over_r)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    build_terms(b, r0, w0, s0, r_c, t);
    for (int i = 0; i < n; ++i) {
        if (F) F[i] = far_F(t, r[i]);
        if (dF_over_r) dF_over_r[i] = far_dF_over_r(t, r[i]);
    }
    free(t);
}

void or_far_fhat(double b, double r0, double w0, double s0, double r_c, int n_terms,
                 int n, const double* k, double* out)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    build_terms(b, r0, w0, s0, r_c, t);
    for (int i = 0; i < n; ++i) out[i] = far_Fhat(t, k[i], n_terms);
    free(t);
}

static double wrap1(double x, double L)
{
    double w = x - L * floor(x / L);
    if (w >= L) w -= L;
    if (w < 0.0) w += L;
    return w;
}

static double minimg(double d, double L)
{
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

/*
 * Near part (Eq. 20) by direct summation over every source atom and every
 * periodic image within r_c.  Targets: targets[0..nt) (NULL = all atoms).
 * Outputs per target: phi[t] = sum q_j N(r), f[3t..] = force on the target.
 */
int or_near(double b, double r0, double w0, double s0, double r_c, const double* box,
            int n, const double* pos, const double* q, int nt, const int* targets,
            double* phi, double* f)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    if (!t) return -1;
    build_terms(b, r0, w0, s0, r_c, t);
    double* w = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!w) { free(t); return -1; }
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) w[3 * i + a] = wrap1(pos[3 * i + a], box[a]);
    int M[3];
    for (int a = 0; a < 3; ++a) M[a] = (r_c < 0.5 * box[a]) ? 0 : (int)ceil(r_c / box[a]);
    double rc2 = r_c * r_c;
    if (targets == NULL) nt = n;

#pragma omp parallel for schedule(dynamic, 16)
    for (int ti = 0; ti < nt; ++ti) {
        int i = targets ? targets[ti] : ti;
        double xi = w[3 * i], yi = w[3 * i + 1], zi = w[3 * i + 2];
        double p = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int j = 0; j < n; ++j) {
            double dx0 = minimg(xi - w[3 * j], box[0]);
            double dy0 = minimg(yi - w[3 * j + 1], box[1]);
            double dz0 = minimg(zi - w[3 * j + 2], box[2]);
            for (int mx = -M[0]; mx <= M[0]; ++mx)
                for (int my = -M[1]; my <= M[1]; ++my)
                    for (int mz = -M[2]; mz <= M[2]; ++mz) {
                        if (i == j && mx == 0 && my == 0 && mz == 0) continue;
                        double dx = dx0 + mx * box[0], dy = dy0 + my * box[1], dz = dz0 + mz * box[2];
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 >= rc2) continue;
                        double r = sqrt(r2);
                        double Fv = 0.0, dFr = 0.0;
                        for (int k = t->n - 1; k >= 0; --k) {
                            double s2 = t->s[k] * t->s[k];
                            double v = t->a[k] * exp(-r2 / (2.0 * s2));
                            Fv += v;
                            dFr -= v / s2;
                        }
                        double Nr = 1.0 / r - Fv;
                        /* -dN/dr / r = 1/r^3 + F'(r)/r */
                        double g = 1.0 / (r2 * r) + dFr;
                        p += q[j] * Nr;
                        fx += q[j] * g * dx;
                        fy += q[j] * g * dy;
                        fz += q[j] * g * dz;
                    }
        }
        phi[ti] = p;
        f[3 * ti] = q[i] * fx;
        f[3 * ti + 1] = q[i] * fy;
        f[3 * ti + 2] = q[i] * fz;
    }
    free(w);
    free(t);
    return 0;
}

/* ---------------------------------------------------------------- k-space */

typedef struct {
    int nk;          /* number of half-space k vectors */
    int ncol;        /* number of (mx, my) columns */
    int *col_mx, *col_my, *col_mz0, *col_len, *col_off;
    int M[3];
} kset;

static void kset_free(kset* K)
{
    free(K->col_mx); free(K->col_my); free(K->col_mz0); free(K->col_len); free(K->col_off);
}

/* Half space of reciprocal vectors 2 pi m / L, m != 0, |k| <= kmax. */
static int kset_build(const double* box, double kmax, kset* K)
{
    for (int a = 0; a < 3; ++a) K->M[a] = (int)floor(kmax * box[a] / (2.0 * M_PI));
    int maxcol = (K->M[0] + 1) * (2 * K->M[1] + 1);
    K->col_mx = (int*)malloc(sizeof(int) * maxcol);
    K->col_my = (int*)malloc(sizeof(int) * maxcol);
    K->col_mz0 = (int*)malloc(sizeof(int) * maxcol);
    K->col_len = (int*)malloc(sizeof(int) * maxcol);
    K->col_off = (int*)malloc(sizeof(int) * maxcol);
    if (!K->col_mx || !K->col_my || !K->col_mz0 || !K->col_len || !K->col_off) return -1;
    int nc = 0, nk = 0;
    double k2max = kmax * kmax;
    for (int mx = 0; mx <= K->M[0]; ++mx)
        for (int my = -K->M[1]; my <= K->M[1]; ++my) {
            if (mx == 0 && my < 0) continue;
            double kx = 2.0 * M_PI * mx / box[0], ky = 2.0 * M_PI * my / box[1];
            double rem = k2max - kx * kx - ky * ky;
            if (rem < 0.0) continue;
            int mzmax = (int)floor(sqrt(rem) * box[2] / (2.0 * M_PI));
            if (mzmax > K->M[2]) mzmax = K->M[2];
            int mz0 = (mx == 0 && my == 0) ? 1 : -mzmax;
            int len = mzmax - mz0 + 1;
            if (len <= 0) continue;
            K->col_mx[nc] = mx; K->col_my[nc] = my; K->col_mz0[nc] = mz0;
            K->col_len[nc] = len; K->col_off[nc] = nk;
            nk += len; ++nc;
        }
    K->ncol = nc;
    K->nk = nk;
    return 0;
}

/* exp(i 2 pi m x / L) for m = 0..M (cx, sx arrays of length M+1). */
static void phases(double x, double L, int M, double* c, double* s)
{
    for (int m = 0; m <= M; ++m) {
        double th = 2.0 * M_PI * (double)m * x / L;
        c[m] = cos(th);
        s[m] = sin(th);
    }
}

/*
 * Far part, exact in k-space (Eqs. 4, 9, F1 with the Gaussians of App. C).
 * n_terms <= 0: every Gaussian of the series; otherwise the first n_terms.
 * kmax: largest |k| summed (<= 0: 9.2 / min_j s_j, where the narrowest
 * Gaussian's transform is below 1e-18 of its peak).
 * Outputs: E_far (includes each charge's interaction with its own far
 * Gaussian; the self term removes it), and per target phi_far, f_far.
 */
int or_far(double b, double r0, double w0, double s0, double r_c, const double* box,
           int n_terms, double kmax, int n, const double* pos, const double* q,
           int nt, const int* targets, double* phi, double* f, double* E_far, int* nk_out)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    if (!t) return -1;
    build_terms(b, r0, w0, s0, r_c, t);
    if (kmax <= 0.0) {
        double smin = t->s[0];
        for (int j = 1; j < t->n; ++j) if (t->s[j] < smin) smin = t->s[j];
        kmax = 9.2 / smin;
    }
    kset K;
    if (kset_build(box, kmax, &K)) { free(t); return -1; }
    int nk = K.nk;
    if (nk_out) *nk_out = nk;
    double V = box[0] * box[1] * box[2];
    double* fh = (double*)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    double* kv = (double*)malloc(sizeof(double) * 3 * (size_t)(nk > 0 ? nk : 1));
    double* Sre = (double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(double));
    double* Sim = (double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(double));
    if (!fh || !kv || !Sre || !Sim) { free(t); return -1; }
    for (int c = 0; c < K.ncol; ++c)
        for (int l = 0; l < K.col_len[c]; ++l) {
            int idx = K.col_off[c] + l;
            double kx = 2.0 * M_PI * K.col_mx[c] / box[0];
            double ky = 2.0 * M_PI * K.col_my[c] / box[1];
            double kz = 2.0 * M_PI * (K.col_mz0[c] + l) / box[2];
            kv[3 * idx] = kx; kv[3 * idx + 1] = ky; kv[3 * idx + 2] = kz;
            fh[idx] = far_Fhat(t, sqrt(kx * kx + ky * ky + kz * kz), n_terms);
        }
    int Mx = K.M[0], My = K.M[1], Mz = K.M[2];

    /* structure factor S(k) = sum_j q_j e^{i k . r_j} */
#pragma omp parallel
    {
        double* sre = (double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(double));
        double* sim = (double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(double));
        double *cx = (double*)malloc(sizeof(double) * (Mx + 1)), *sx = (double*)malloc(sizeof(double) * (Mx + 1));
        double *cy = (double*)malloc(sizeof(double) * (My + 1)), *sy = (double*)malloc(sizeof(double) * (My + 1));
        double *cz = (double*)malloc(sizeof(double) * (2 * Mz + 1)), *sz = (double*)malloc(sizeof(double) * (2 * Mz + 1));
        double *tc = (double*)malloc(sizeof(double) * (Mz + 1)), *ts = (double*)malloc(sizeof(double) * (Mz + 1));
#pragma omp for schedule(static)
        for (int j = 0; j < n; ++j) {
            phases(pos[3 * j], box[0], Mx, cx, sx);
            phases(pos[3 * j + 1], box[1], My, cy, sy);
            phases(pos[3 * j + 2], box[2], Mz, tc, ts);
            for (int m = 0; m <= Mz; ++m) {
                cz[Mz + m] = tc[m]; sz[Mz + m] = ts[m];
                cz[Mz - m] = tc[m]; sz[Mz - m] = -ts[m];
            }
            double qj = q[j];
            for (int c = 0; c < K.ncol; ++c) {
                int mx = K.col_mx[c], my = K.col_my[c];
                double ycr = cy[my < 0 ? -my : my], yci = (my < 0 ? -sy[-my] : sy[my]);
                /* e^{i(kx x + ky y)} */
                double ar = cx[mx] * ycr - sx[mx] * yci;
                double ai = cx[mx] * yci + sx[mx] * ycr;
                ar *= qj; ai *= qj;
                int off = K.col_off[c], mz0 = K.col_mz0[c], len = K.col_len[c];
                const double* czp = cz + Mz + mz0;
                const double* szp = sz + Mz + mz0;
                for (int l = 0; l < len; ++l) {
                    sre[off + l] += ar * czp[l] - ai * szp[l];
                    sim[off + l] += ar * szp[l] + ai * czp[l];
                }
            }
        }
#pragma omp critical
        {
            for (int k = 0; k < nk; ++k) { Sre[k] += sre[k]; Sim[k] += sim[k]; }
        }
        free(sre); free(sim); free(cx); free(sx); free(cy); free(sy); free(cz); free(sz); free(tc); free(ts);
    }

    /* E_far = 1/(2V) sum_{k != 0} Fhat |S|^2 = 1/V sum_{half} Fhat |S|^2 */
    double e = 0.0;
    for (int k = 0; k < nk; ++k) e += fh[k] * (Sre[k] * Sre[k] + Sim[k] * Sim[k]);
    if (E_far) *E_far = e / V;

    if (targets == NULL) nt = n;
#pragma omp parallel
    {
        double *cx = (double*)malloc(sizeof(double) * (Mx + 1)), *sx = (double*)malloc(sizeof(double) * (Mx + 1));
        double *cy = (double*)malloc(sizeof(double) * (My + 1)), *sy = (double*)malloc(sizeof(double) * (My + 1));
        double *cz = (double*)malloc(sizeof(double) * (2 * Mz + 1)), *sz = (double*)malloc(sizeof(double) * (2 * Mz + 1));
        double *tc = (double*)malloc(sizeof(double) * (Mz + 1)), *ts = (double*)malloc(sizeof(double) * (Mz + 1));
#pragma omp for schedule(static)
        for (int ti = 0; ti < nt; ++ti) {
            int i = targets ? targets[ti] : ti;
            phases(pos[3 * i], box[0], Mx, cx, sx);
            phases(pos[3 * i + 1], box[1], My, cy, sy);
            phases(pos[3 * i + 2], box[2], Mz, tc, ts);
            for (int m = 0; m <= Mz; ++m) {
                cz[Mz + m] = tc[m]; sz[Mz + m] = ts[m];
                cz[Mz - m] = tc[m]; sz[Mz - m] = -ts[m];
            }
            double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
            for (int c = 0; c < K.ncol; ++c) {
                int mx = K.col_mx[c], my = K.col_my[c];
                double ycr = cy[my < 0 ? -my : my], yci = (my < 0 ? -sy[-my] : sy[my]);
                double ar = cx[mx] * ycr - sx[mx] * yci;
                double ai = cx[mx] * yci + sx[mx] * ycr;
                int off = K.col_off[c], mz0 = K.col_mz0[c], len = K.col_len[c];
                for (int l = 0; l < len; ++l) {
                    int k = off + l;
                    /* e^{i k.r_i} = (er, ei); S e^{-i k.r_i} = S * conj(e) */
                    double er = ar * cz[Mz + mz0 + l] - ai * sz[Mz + mz0 + l];
                    double ei = ar * sz[Mz + mz0 + l] + ai * cz[Mz + mz0 + l];
                    double re = Sre[k] * er + Sim[k] * ei;
                    double im = Sim[k] * er - Sre[k] * ei;
                    p += fh[k] * re;
                    double w = fh[k] * im;
                    gx += w * kv[3 * k];
                    gy += w * kv[3 * k + 1];
                    gz += w * kv[3 * k + 2];
                }
            }
            phi[ti] = 2.0 * p / V;
            f[3 * ti] = -2.0 * q[i] * gx / V;
            f[3 * ti + 1] = -2.0 * q[i] * gy / V;
            f[3 * ti + 2] = -2.0 * q[i] * gz / V;
        }
        free(cx); free(sx); free(cy); free(sy); free(cz); free(sz); free(tc); free(ts);
    }
    free(fh); free(kv); free(Sre); free(Sim);
    kset_free(&K);
    free(t);
    return 0;
}

/* F(0) of the full series (the self-interaction constant of Eq. 10's self term). */
double or_F0(double b, double r0, double w0, double s0, double r_c)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    build_terms(b, r0, w0, s0, r_c, t);
    double v = 0.0;
    for (int j = t->n - 1; j >= 0; --j) v += t->a[j];
    free(t);
    return v;
}

/*
 * Far part as a real-space periodic image sum of the first n_terms Gaussians
 * (Poisson-summation partner of or_far with the same n_terms).  The i == j,
 * n = 0 term is included, like in or_far.  Images out to 10 widths of the
 * widest kept Gaussian.  For tiny systems only.
 */
int or_far_realspace(double b, double r0, double w0, double s0, double r_c, const double* box,
                     int n_terms, int n, const double* pos, const double* q,
                     double* phi, double* f, double* E_far)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    if (!t) return -1;
    build_terms(b, r0, w0, s0, r_c, t);
    int nterm = (n_terms > 0 && n_terms < t->n) ? n_terms : t->n;
    double smax = 0.0;
    for (int j = 0; j < nterm; ++j) if (t->s[j] > smax) smax = t->s[j];
    int M[3];
    for (int a = 0; a < 3; ++a) M[a] = (int)ceil(10.0 * smax / box[a]) + 1;
    double e = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : e)
    for (int i = 0; i < n; ++i) {
        double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int j = 0; j < n; ++j) {
            double dx0 = pos[3 * i] - pos[3 * j];
            double dy0 = pos[3 * i + 1] - pos[3 * j + 1];
            double dz0 = pos[3 * i + 2] - pos[3 * j + 2];
            for (int mx = -M[0]; mx <= M[0]; ++mx)
                for (int my = -M[1]; my <= M[1]; ++my)
                    for (int mz = -M[2]; mz <= M[2]; ++mz) {
                        double dx = dx0 + mx * box[0], dy = dy0 + my * box[1], dz = dz0 + mz * box[2];
                        double r2 = dx * dx + dy * dy + dz * dz;
                        double g = 0.0, h = 0.0;
                        for (int k = 0; k < nterm; ++k) {
                            double s2 = t->s[k] * t->s[k];
                            double v = t->a[k] * exp(-r2 / (2.0 * s2));
                            g += v;
                            h += v / s2;
                        }
                        p += q[j] * g;
                        /* -d/dr_i of q_i q_j g(|d|) = q_i q_j h d */
                        gx += q[j] * h * dx;
                        gy += q[j] * h * dy;
                        gz += q[j] * h * dz;
                    }
        }
        if (phi) phi[i] = p;
        if (f) { f[3 * i] = q[i] * gx; f[3 * i + 1] = q[i] * gy; f[3 * i + 2] = q[i] * gz; }
        e += 0.5 * q[i] * p;
    }
    if (E_far) *E_far = e;
    free(t);
    return 0;
}

/*
 * Full u-series evaluation: E and per-target phi, F (near + far + self).
 * energies[0..3] = E, E_near, E_far, E_self (E_near only when targets == NULL).
 */
int or_eval(double b, double r0, double w0, double s0, double r_c, const double* box,
            int n_terms, double kmax, int n, const double* pos, const double* q,
            int nt, const int* targets, double* phi, double* f,
            double* phi_near, double* f_near, double* phi_far, double* f_far, double* energies)
{
    if (targets == NULL) nt = n;
    size_t m = (size_t)(nt > 0 ? nt : 1);
    double* pn = phi_near ? phi_near : (double*)malloc(sizeof(double) * m);
    double* fn = f_near ? f_near : (double*)malloc(sizeof(double) * 3 * m);
    double* pf = phi_far ? phi_far : (double*)malloc(sizeof(double) * m);
    double* ff = f_far ? f_far : (double*)malloc(sizeof(double) * 3 * m);
    if (!pn || !fn || !pf || !ff) return -1;
    int rc = or_near(b, r0, w0, s0, r_c, box, n, pos, q, nt, targets, pn, fn);
    double Ef = 0.0;
    if (!rc) rc = or_far(b, r0, w0, s0, r_c, box, n_terms, kmax, n, pos, q, nt, targets, pf, ff, &Ef, NULL);
    double F0 = or_F0(b, r0, w0, s0, r_c);
    double q2 = 0.0, en = 0.0;
    for (int j = 0; j < n; ++j) q2 += q[j] * q[j];
    for (int ti = 0; ti < nt; ++ti) {
        int i = targets ? targets[ti] : ti;
        phi[ti] = pn[ti] + pf[ti] - F0 * q[i];
        for (int a = 0; a < 3; ++a) f[3 * ti + a] = fn[3 * ti + a] + ff[3 * ti + a];
        en += 0.5 * q[i] * pn[ti];
    }
    double es = -0.5 * F0 * q2;
    if (energies) {
        energies[1] = targets ? 0.0 : en;
        energies[2] = Ef;
        energies[3] = es;
        energies[0] = energies[1] + Ef + es;
    }
    if (!phi_near) free(pn);
    if (!f_near) free(fn);
    if (!phi_far) free(pf);
    if (!f_far) free(ff);
    return rc;
}

/* ----------------------------------------------------------------- virial */

/* sum_j s_j^2 Fhat_j(k): the strain derivative weight of the far part. */
static double far_Fhat_s2(const or_terms* t, double k, int nk)
{
    int n = (nk > 0 && nk < t->n) ? nk : t->n;
    double sum = 0.0;
    for (int j = 0; j < n; ++j) {
        double s2 = t->s[j] * t->s[j];
        double x = 0.5 * s2 * k * k;
        if (x > 745.0) continue;
        sum += s2 * t->a[j] * pow(2.0 * M_PI * s2, 1.5) * exp(-x);
    }
    return sum;
}

/*
 * Virial tensor W = -dE/d(strain) under an affine strain of positions and box
 * (row-major 3 x 3, symmetric).
 *   near:  W = 1/2 sum_{i != j, images, r < r_c} d (x) f_ij,  f_ij = q_i q_j (1/r^3 + F'(r)/r) d
 *          (the pair force of Eq. 20's near function on i, d = r_i - r_j - image)
 *   far:   W_ab = delta_ab E_far - (1/2V) sum_{k != 0} |S(k)|^2 k_a k_b sum_j s_j^2 Fhat_j(k)
 *          (the strain derivative of Eq. F1: V grows with the trace, k shrinks as the box grows,
 *           and dFhat_j/d(k^2) = -s_j^2 Fhat_j / 2)
 *   self:  no box dependence (F(0) is fixed by sigma), no contribution.
 * n_terms / kmax as in or_far.
 */
int or_virial(double b, double r0, double w0, double s0, double r_c, const double* box,
              int n_terms, double kmax, int n, const double* pos, const double* q,
              double* W_near, double* W_far)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    if (!t) return -1;
    build_terms(b, r0, w0, s0, r_c, t);
    /* near: direct pair sum */
    double* w = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!w) { free(t); return -1; }
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) w[3 * i + a] = wrap1(pos[3 * i + a], box[a]);
    int M[3];
    for (int a = 0; a < 3; ++a) M[a] = (r_c < 0.5 * box[a]) ? 0 : (int)ceil(r_c / box[a]);
    double rc2 = r_c * r_c;
    double wn[6] = {0, 0, 0, 0, 0, 0};   /* xx yy zz xy xz yz */
#pragma omp parallel
    {
        double loc[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                double dx0 = minimg(w[3 * i] - w[3 * j], box[0]);
                double dy0 = minimg(w[3 * i + 1] - w[3 * j + 1], box[1]);
                double dz0 = minimg(w[3 * i + 2] - w[3 * j + 2], box[2]);
                for (int mx = -M[0]; mx <= M[0]; ++mx)
                    for (int my = -M[1]; my <= M[1]; ++my)
                        for (int mz = -M[2]; mz <= M[2]; ++mz) {
                            if (i == j && mx == 0 && my == 0 && mz == 0) continue;
                            double dx = dx0 + mx * box[0], dy = dy0 + my * box[1], dz = dz0 + mz * box[2];
                            double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 >= rc2) continue;
                            double r = sqrt(r2), dFr = 0.0;
                            for (int k = t->n - 1; k >= 0; --k) {
                                double s2 = t->s[k] * t->s[k];
                                dFr -= t->a[k] * exp(-r2 / (2.0 * s2)) / s2;
                            }
                            double g = 0.5 * q[i] * q[j] * (1.0 / (r2 * r) + dFr);
                            loc[0] += g * dx * dx; loc[1] += g * dy * dy; loc[2] += g * dz * dz;
                            loc[3] += g * dx * dy; loc[4] += g * dx * dz; loc[5] += g * dy * dz;
                        }
            }
        }
#pragma omp critical
        for (int c = 0; c < 6; ++c) wn[c] += loc[c];
    }
    free(w);
    /* far: k-space */
    if (kmax <= 0.0) {
        double smin = t->s[0];
        for (int j = 1; j < t->n; ++j) if (t->s[j] < smin) smin = t->s[j];
        kmax = 9.2 / smin;
    }
    kset K;
    if (kset_build(box, kmax, &K)) { free(t); return -1; }
    double V = box[0] * box[1] * box[2];
    double ef = 0.0, wf[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel
    {
        double le = 0.0, lw[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 4)
        for (int c = 0; c < K.ncol; ++c) {
            double kx = 2.0 * M_PI * K.col_mx[c] / box[0];
            double ky = 2.0 * M_PI * K.col_my[c] / box[1];
            for (int l = 0; l < K.col_len[c]; ++l) {
                double kz = 2.0 * M_PI * (K.col_mz0[c] + l) / box[2];
                double sr = 0.0, si = 0.0;
                for (int j = 0; j < n; ++j) {
                    double th = kx * pos[3 * j] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
                    sr += q[j] * cos(th);
                    si += q[j] * sin(th);
                }
                double S2 = sr * sr + si * si;
                double kk = sqrt(kx * kx + ky * ky + kz * kz);
                le += far_Fhat(t, kk, n_terms) * S2;
                double u = far_Fhat_s2(t, kk, n_terms) * S2;
                lw[0] += u * kx * kx; lw[1] += u * ky * ky; lw[2] += u * kz * kz;
                lw[3] += u * kx * ky; lw[4] += u * kx * kz; lw[5] += u * ky * kz;
            }
        }
#pragma omp critical
        {
            ef += le;
            for (int c = 0; c < 6; ++c) wf[c] += lw[c];
        }
    }
    kset_free(&K);
    ef /= V;                              /* half space: (1/2V) sum_all = (1/V) sum_half */
    for (int c = 0; c < 6; ++c) wf[c] = -wf[c] / V;
    wf[0] += ef; wf[1] += ef; wf[2] += ef;
    const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
    for (int e = 0; e < 9; ++e) {
        if (W_near) W_near[e] = wn[map[e]];
        if (W_far) W_far[e] = wf[map[e]];
    }
    free(t);
    return 0;
}

/*
 * Far-part virial as a real-space image sum of the first n_terms Gaussians:
 * W = 1/2 sum_{i, j, images} q_i q_j h(|d|) d (x) d, h = sum_j a_j e^{-d^2/2 s_j^2} / s_j^2.
 * For a neutral system this is the Poisson-summation partner of or_virial's far
 * part (the k = 0 term is zero).  Tiny systems only.
 */
int or_far_virial_realspace(double b, double r0, double w0, double s0, double r_c, const double* box,
                            int n_terms, int n, const double* pos, const double* q, double* W_far)
{
    or_terms* t = (or_terms*)malloc(sizeof(or_terms));
    if (!t) return -1;
    build_terms(b, r0, w0, s0, r_c, t);
    int nterm = (n_terms > 0 && n_terms < t->n) ? n_terms : t->n;
    double smax = 0.0;
    for (int j = 0; j < nterm; ++j) if (t->s[j] > smax) smax = t->s[j];
    int M[3];
    for (int a = 0; a < 3; ++a) M[a] = (int)ceil(10.0 * smax / box[a]) + 1;
    double wf[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel
    {
        double loc[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double dx0 = pos[3 * i] - pos[3 * j];
                double dy0 = pos[3 * i + 1] - pos[3 * j + 1];
                double dz0 = pos[3 * i + 2] - pos[3 * j + 2];
                for (int mx = -M[0]; mx <= M[0]; ++mx)
                    for (int my = -M[1]; my <= M[1]; ++my)
                        for (int mz = -M[2]; mz <= M[2]; ++mz) {
                            double dx = dx0 + mx * box[0], dy = dy0 + my * box[1], dz = dz0 + mz * box[2];
                            double r2 = dx * dx + dy * dy + dz * dz;
                            double h = 0.0;
                            for (int k = 0; k < nterm; ++k) {
                                double s2 = t->s[k] * t->s[k];
                                h += t->a[k] * exp(-r2 / (2.0 * s2)) / s2;
                            }
                            double g = 0.5 * q[i] * q[j] * h;
                            loc[0] += g * dx * dx; loc[1] += g * dy * dy; loc[2] += g * dz * dz;
                            loc[3] += g * dx * dy; loc[4] += g * dx * dz; loc[5] += g * dy * dz;
                        }
            }
#pragma omp critical
        for (int c = 0; c < 6; ++c) wf[c] += loc[c];
    }
    const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
    for (int e = 0; e < 9; ++e) W_far[e] = wf[map[e]];
    free(t);
    return 0;
}

/* ------------------------------------------------------------------ Ewald */

/*
 * Classic Ewald sum (Eqs. 6-10) with splitting width sigma_e: real-space
 * erfc(r / (sqrt2 sigma_e)) / r out to rcut (all images), k-space out to kmax,
 * self term -sum q^2 / sqrt(2 pi sigma_e^2).  Independent of the u-series
 * code above; used to pin it.  energies[0..2] = total, real, reciprocal+self.
 */
int or_ewald(const double* box, double sigma_e, double rcut, double kmax,
             int n, const double* pos, const double* q, double* phi, double* f, double* energies)
{
    int M[3];
    for (int a = 0; a < 3; ++a) M[a] = (int)ceil(rcut / box[a]) + 1;
    double V = box[0] * box[1] * box[2];
    double rc2 = rcut * rcut;
    double a2 = 1.0 / (sqrt(2.0) * sigma_e);
    double er = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : er)
    for (int i = 0; i < n; ++i) {
        double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int j = 0; j < n; ++j) {
            double dx0 = pos[3 * i] - pos[3 * j];
            double dy0 = pos[3 * i + 1] - pos[3 * j + 1];
            double dz0 = pos[3 * i + 2] - pos[3 * j + 2];
            for (int mx = -M[0]; mx <= M[0]; ++mx)
                for (int my = -M[1]; my <= M[1]; ++my)
                    for (int mz = -M[2]; mz <= M[2]; ++mz) {
                        if (i == j && mx == 0 && my == 0 && mz == 0) continue;
                        double dx = dx0 + mx * box[0], dy = dy0 + my * box[1], dz = dz0 + mz * box[2];
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 >= rc2) continue;
                        double r = sqrt(r2);
                        double v = erfc(a2 * r) / r;
                        /* -d/dr [erfc(a r)/r] = erfc(a r)/r^2 + 2a/sqrt(pi) e^{-a^2 r^2} / r */
                        double g = (v + 2.0 * a2 / sqrt(M_PI) * exp(-a2 * a2 * r2)) / r2;
                        p += q[j] * v;
                        gx += q[j] * g * dx; gy += q[j] * g * dy; gz += q[j] * g * dz;
                    }
        }
        phi[i] = p;
        f[3 * i] = q[i] * gx; f[3 * i + 1] = q[i] * gy; f[3 * i + 2] = q[i] * gz;
        er += 0.5 * q[i] * p;
    }
    /* reciprocal part: direct cos/sin per (k, atom), full sphere without k = 0 */
    int K[3];
    for (int a = 0; a < 3; ++a) K[a] = (int)floor(kmax * box[a] / (2.0 * M_PI));
    double ek = 0.0;
    double* pk = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* fk = (double*)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    for (int mx = -K[0]; mx <= K[0]; ++mx)
        for (int my = -K[1]; my <= K[1]; ++my)
            for (int mz = -K[2]; mz <= K[2]; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                double kx = 2.0 * M_PI * mx / box[0], ky = 2.0 * M_PI * my / box[1], kz = 2.0 * M_PI * mz / box[2];
                double k2 = kx * kx + ky * ky + kz * kz;
                if (k2 > kmax * kmax) continue;
                double A = 4.0 * M_PI / k2 * exp(-0.5 * sigma_e * sigma_e * k2);
                double sr = 0.0, si = 0.0;
                for (int j = 0; j < n; ++j) {
                    double th = kx * pos[3 * j] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
                    sr += q[j] * cos(th);
                    si += q[j] * sin(th);
                }
                ek += A * (sr * sr + si * si);
#pragma omp parallel for schedule(static)
                for (int i = 0; i < n; ++i) {
                    double th = kx * pos[3 * i] + ky * pos[3 * i + 1] + kz * pos[3 * i + 2];
                    double c = cos(th), s = sin(th);
                    /* Re(S e^{-i th}) and Im(S e^{-i th}) */
                    double re = sr * c + si * s;
                    double im = si * c - sr * s;
                    pk[i] += A * re;
                    fk[3 * i] += A * im * kx; fk[3 * i + 1] += A * im * ky; fk[3 * i + 2] += A * im * kz;
                }
            }
    ek /= 2.0 * V;
    double q2 = 0.0;
    for (int j = 0; j < n; ++j) q2 += q[j] * q[j];
    double es = -q2 / sqrt(2.0 * M_PI * sigma_e * sigma_e);
    for (int i = 0; i < n; ++i) {
        phi[i] += pk[i] / V - 2.0 * q[i] / sqrt(2.0 * M_PI * sigma_e * sigma_e);
        for (int a = 0; a < 3; ++a) f[3 * i + a] += -q[i] * fk[3 * i + a] / V;
    }
    free(pk); free(fk);
    if (energies) { energies[1] = er; energies[2] = ek + es; energies[0] = er + ek + es; }
    return 0;
}

/* ------------------------------------------- single-precision cell predicate */

/*
 * The cell list is defined in single precision so that two independent
 * implementations can agree on it bit for bit.  Per axis (box length L,
 * nc cells), with RN rounding and no contraction:
 *     invL = (float)(1/L), Lf = (float)L, cs = (float)(nc / L)
 *     k  = floorf(x * invL)
 *     xw = fmaf(-k, Lf, x);  if (xw < 0) xw += Lf;  if (xw >= Lf) xw -= Lf;
 *     c  = (int)(xw * cs) clamped to [0, nc-1]
 * Non-finite coordinates give xw = 0, c = 0.  The cell id is
 * (cz * ncy + cy) * ncx + cx.
 * A pair (i, j != i) is listed when j lies in one of the 27 cells adjacent to
 * i's cell (periodically; nc >= 3 on every axis) and, with the periodic
 * shift sh = -Lf, 0 or +Lf chosen by that cell offset,
 *     d = (xw_j + sh) - xw_i  (per axis, two RN roundings)
 *     r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < (float)(r_c * r_c).
 */
static float canon_wrap(float x, float invL, float Lf)
{
    if (!isfinite(x)) return 0.0f;
    float k = floorf(x * invL);
    float xw = fmaf(-k, Lf, x);
    if (xw < 0.0f) xw += Lf;
    if (xw >= Lf) xw -= Lf;
    return xw;
}

static int canon_cell(float xw, float cs, int nc)
{
    float u = xw * cs;
    int c = (u >= 0.0f) ? (int)u : 0;
    if (c > nc - 1) c = nc - 1;
    return c;
}

void or_canon_cells(int n, const float* xyzq, const double* box, const int* nc, int* cell, float* xw)
{
    float invL[3], Lf[3], cs[3];
    for (int a = 0; a < 3; ++a) {
        invL[a] = (float)(1.0 / box[a]);
        Lf[a] = (float)box[a];
        cs[a] = (float)((double)nc[a] / box[a]);
    }
    for (int i = 0; i < n; ++i) {
        int ci[3];
        int bad = !(isfinite(xyzq[4 * i]) && isfinite(xyzq[4 * i + 1]) && isfinite(xyzq[4 * i + 2]));
        for (int a = 0; a < 3; ++a) {
            float w = bad ? 0.0f : canon_wrap(xyzq[4 * i + a], invL[a], Lf[a]);
            if (xw) xw[3 * i + a] = w;
            ci[a] = canon_cell(w, cs[a], nc[a]);
        }
        cell[i] = (ci[2] * nc[1] + ci[1]) * nc[0] + ci[0];
    }
}

/* splitmix64 finaliser (Steele, Lea, Flood 2014), used as an order-free set hash. */
static uint64_t mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Per atom: the number of listed partners and the wrap-around sum of
 * mix64(j) over them (j = caller index).  Uses its own cell membership lists.
 */
int or_canon_pairs(int n, const float* xyzq, const double* box, const int* nc, double r_c,
                   int* count, uint64_t* hash)
{
    int ncell = nc[0] * nc[1] * nc[2];
    int* cell = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    float* xw = (float*)malloc(sizeof(float) * 3 * (size_t)(n > 0 ? n : 1));
    int* head = (int*)malloc(sizeof(int) * (size_t)ncell);
    int* next = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!cell || !xw || !head || !next) return -1;
    or_canon_cells(n, xyzq, box, nc, cell, xw);
    for (int c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = n - 1; i >= 0; --i) { next[i] = head[cell[i]]; head[cell[i]] = i; }
    float Lf[3];
    for (int a = 0; a < 3; ++a) Lf[a] = (float)box[a];
    float rc2 = (float)(r_c * r_c);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        int c = cell[i];
        int cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / (nc[0] * nc[1]);
        int cnt = 0;
        uint64_t h = 0;
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    int o[3] = {ox, oy, oz}, cc[3] = {cx, cy, cz}, nn[3];
                    float sh[3];
                    for (int a = 0; a < 3; ++a) {
                        int v = cc[a] + o[a];
                        sh[a] = 0.0f;
                        if (v < 0) { v += nc[a]; sh[a] = -Lf[a]; }
                        else if (v >= nc[a]) { v -= nc[a]; sh[a] = Lf[a]; }
                        nn[a] = v;
                    }
                    int nb = (nn[2] * nc[1] + nn[1]) * nc[0] + nn[0];
                    for (int j = head[nb]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        float dx = (xw[3 * j] + sh[0]) - xw[3 * i];
                        float dy = (xw[3 * j + 1] + sh[1]) - xw[3 * i + 1];
                        float dz = (xw[3 * j + 2] + sh[2]) - xw[3 * i + 2];
                        float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        if (r2 < rc2) { ++cnt; h += mix64((uint64_t)j); }
                    }
                }
        count[i] = cnt;
        hash[i] = h;
    }
    free(cell); free(xw); free(head); free(next);
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
