/*
 * FP64 CPU oracle for multi-layer collimated-beam MBIR.
 *
 * TEST INFRASTRUCTURE ONLY (see mbir_oracle.h).  Plain loops in double
 * precision, following the paper's Section 2 in its own order:
 *   - travel time of a leg by binary search on the incident angle theta_1
 *     (eq. 4, 5, 6);
 *   - attenuated, windowed pulse h~(gamma, t) (eq. 9, 10) tabulated once on a
 *     (gamma, tau) grid and read back by bilinear interpolation;
 *   - the apodized per-pair model (eq. 12, 13) summed over voxels (eq. 11);
 *   - direct arrivals (eq. 1) eliminated by projection;
 *   - the QGGMRF prior with spatially varying scale (eq. 14-17);
 *   - the MAP cost of eq. 18 minimised by a fixed majorize-minimize
 *     conjugate-gradient iteration, or by coloured iterative coordinate
 *     descent (the paper's ICD).
 * OpenMP pragmas only split independent loops across threads; they change no
 * arithmetic.
 */
#include "mbir_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* pulse: Gaussian-modulated cosine with an n_cycles-period FWHM envelope */
/* ------------------------------------------------------------------ */
static double pulse_sigma(const orc_geom* g)
{
    return g->n_cycles / (2.0 * sqrt(2.0 * log(2.0)) * g->fc);
}

int orc_pulse_support(const orc_geom* g)
{
    /* t0 of eq. 10: eight envelope standard deviations, whole samples */
    return (int)ceil(8.0 * pulse_sigma(g) * g->fs);
}

double orc_pulse(const orc_geom* g, double t)
{
    double sg = pulse_sigma(g);
    double tc = 0.5 * orc_pulse_support(g) / g->fs;
    double u = t - tc;
    return exp(-u * u / (2.0 * sg * sg)) * cos(2.0 * M_PI * g->fc * u);
}

/* ------------------------------------------------------------------ */
/* layer split of a voxel depth                                        */
/* ------------------------------------------------------------------ */
/* eta[l] = thickness of each layer crossed above depth z, and the part of the
 * voxel's own layer above it.  Returns the number of layers with eta > 0
 * (the voxel layer index + 1, or the index when the voxel sits on its top). */
static int layer_split(const orc_geom* g, double z, double* eta, int* lv_out)
{
    double top = 0.0;
    int lv = 0;
    for (int l = 0; l < g->n_layers; ++l) {
        if (l == g->n_layers - 1 || z < top + g->thickness[l]) { lv = l; break; }
        top += g->thickness[l];
    }
    for (int l = 0; l < lv; ++l) eta[l] = g->thickness[l];
    eta[lv] = z - top;
    if (lv_out) *lv_out = lv;
    return eta[lv] > 0.0 ? lv + 1 : lv;
}

double orc_transmission(const orc_geom* g, double z)
{
    double eta[ORC_MAX_LAYERS];
    int lv;
    layer_split(g, z, eta, &lv);
    double tau = 1.0;
    for (int l = 1; l <= lv; ++l) {
        double z1 = g->density[l - 1] * g->speed[l - 1];
        double z2 = g->density[l] * g->speed[l];
        tau *= 4.0 * z1 * z2 / ((z1 + z2) * (z1 + z2));
    }
    return tau;
}

/* angles of eq. 6 from the incident angle theta_1; returns 0 when a layer is
 * past its critical angle (the height of eq. 5 is then infinite) */
static int snell_angles(const orc_geom* g, int nl, double theta1, double* th)
{
    th[0] = theta1;
    for (int k = 1; k < nl; ++k) {
        double s = sin(th[k - 1]) * g->speed[k] / g->speed[k - 1];
        if (!(s < 1.0)) return 0;
        th[k] = asin(s);
    }
    return 1;
}

/* lateral reach of eq. 5 for a given theta_1 */
static double leg_height(const orc_geom* g, int nl, const double* eta, double theta1)
{
    double th[ORC_MAX_LAYERS];
    if (!snell_angles(g, nl, theta1, th)) return INFINITY;
    double hsum = 0.0;
    for (int l = 0; l < nl; ++l) hsum += eta[l] * tan(th[l]);
    return hsum;
}

void orc_leg(const orc_geom* g, double h, double z,
             double* T, double* gamma, double* Theta, double* theta1_out)
{
    double eta[ORC_MAX_LAYERS];
    int nl = layer_split(g, z, eta, NULL);
    h = fabs(h);
    double cmax = 0.0;
    for (int l = 0; l < nl; ++l) if (g->speed[l] > cmax) cmax = g->speed[l];
    /* the height grows without bound as the fastest crossed layer reaches 90
     * degrees, so the binary search runs over [0, theta_crit) */
    double hi = (g->speed[0] >= cmax) ? 0.5 * M_PI : asin(g->speed[0] / cmax);
    double lo = 0.0;
    double theta1 = 0.0;
    if (h > 0.0 && nl > 0) {
        for (int it = 0; it < 400; ++it) {
            double mid = lo + 0.5 * (hi - lo);
            if (mid <= lo || mid >= hi) break;
            if (leg_height(g, nl, eta, mid) < h) lo = mid; else hi = mid;
        }
        theta1 = lo + 0.5 * (hi - lo);
    }
    double th[ORC_MAX_LAYERS];
    snell_angles(g, nl, theta1, th);
    double t = 0.0, gm = 0.0, sum_th = 0.0;
    for (int l = 0; l < nl; ++l) {
        double zl = eta[l] * tan(th[l]);            /* z_{i,l} of eq. 4 */
        double path = sqrt(zl * zl + eta[l] * eta[l]);
        t += path / g->speed[l];                     /* eq. 4 */
        gm += g->atten[l] * path;                    /* gamma_l = c_l alpha_l T_l */
        sum_th += th[l];
    }
    *T = t;
    *gamma = gm;
    *Theta = sum_th;
    if (theta1_out) *theta1_out = theta1;
}

/* ------------------------------------------------------------------ */
/* attenuated pulse family h(gamma, t), eq. 9                          */
/* ------------------------------------------------------------------ */
double orc_gamma_max(const orc_geom* g)
{
    if (g->gamma_max > 0.0) return g->gamma_max;
    /* default: twice the two-way vertical loss down to the deepest pixel */
    double zb = g->z0 + (g->img_h - 0.5) * g->pitch;
    double eta[ORC_MAX_LAYERS];
    int nl = layer_split(g, zb, eta, NULL);
    double s = 0.0;
    for (int l = 0; l < nl; ++l) s += g->atten[l] * eta[l];
    return 4.0 * s;
}

int orc_effective_G(const orc_geom* g)
{
    return orc_gamma_max(g) > 0.0 ? g->G : 1;
}

/* 16-point Gauss-Legendre nodes on [-1, 1] by Newton's method on P_16 */
static void gauss_legendre16(double* xn, double* wn)
{
    const int n = 16;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        xn[i] = x;
        wn[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

/* h(gamma, tau) = int S(f) e^{-gamma |f|} e^{2 pi i f tau} df, with S the
 * spectrum of the pulse: for the Gaussian-modulated cosine centred at t_c,
 * S(f) = e^{-2 pi i f t_c} sigma sqrt(2 pi)/2 [G(f - fc) + G(f + fc)],
 * G(u) = exp(-2 pi^2 sigma^2 u^2).  The even bracket folds the integral onto
 * f >= 0.  Composite 16-point Gauss-Legendre quadrature on f in [0, F];
 * panels_scale > 1 refines the panels (used to check convergence). */
void orc_pulse_table(const orc_geom* g, double* tab, int panels_scale)
{
    int Tw = orc_pulse_support(g);
    int nq = g->Q * Tw + 1;
    int G = orc_effective_G(g);
    double gmax = orc_gamma_max(g);
    double sg = pulse_sigma(g);
    double sf = 1.0 / (2.0 * M_PI * sg);
    double t0 = Tw / g->fs;
    double tc = 0.5 * t0;
    double F = g->fc + 16.0 * sf;
    double pw = fmin(0.5 * sf, 0.25 / t0) / (panels_scale > 0 ? panels_scale : 1);
    int np = (int)ceil(F / pw);
    pw = F / np;
    double xn[16], wn[16];
    gauss_legendre16(xn, wn);
    int nf = np * 16;
    double* f = (double*)malloc(sizeof(double) * nf);
    double* sw = (double*)malloc(sizeof(double) * nf);
    for (int p = 0; p < np; ++p)
        for (int i = 0; i < 16; ++i) {
            double fv = (p + 0.5) * pw + 0.5 * pw * xn[i];
            double a = fv - g->fc, b = fv + g->fc;
            double spec = exp(-2.0 * M_PI * M_PI * sg * sg * a * a) +
                          exp(-2.0 * M_PI * M_PI * sg * sg * b * b);
            f[p * 16 + i] = fv;
            sw[p * 16 + i] = 0.5 * pw * wn[i] * sg * sqrt(2.0 * M_PI) * spec;
        }
    #pragma omp parallel for schedule(dynamic)
    for (int gi = 0; gi < G; ++gi) {
        double gam = (G > 1) ? gi * gmax / (G - 1) : 0.0;
        for (int q = 0; q < nq; ++q) {
            double tau = q / (g->fs * g->Q);
            double acc = 0.0;
            for (int n = 0; n < nf; ++n)
                acc += sw[n] * exp(-gam * f[n]) * cos(2.0 * M_PI * f[n] * (tau - tc));
            tab[(long)gi * nq + q] = acc;
        }
    }
    free(f);
    free(sw);
}

/* ------------------------------------------------------------------ */
/* plans                                                               */
/* ------------------------------------------------------------------ */
struct orc_plan {
    orc_geom g;
    int Tw, G, nq;
    double gmax, t0;
    double* tab;
    long npix;
    long* pix;            /* pixel index of each slot */
    int npos;
    double* pos;          /* distinct transducer lateral positions (then the tilted Tx, if any) */
    int* pos_tx;          /* 1 for an entry of a tilted transmitter */
    int* tx_pos;          /* n_tx */
    int* rx_pos;          /* n_tx * n_rx */
    double* tau_row;      /* transmission per image row */
    /* per position: legs for every slot (T, gamma, phi); NULL until needed */
    double** leg;
};

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static int find_pos(const double* pos, int n, double v)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (pos[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

orc_plan* orc_plan_create(const orc_geom* g, const long* pix, long npix, int nthreads)
{
    (void)nthreads;
    orc_plan* p = (orc_plan*)calloc(1, sizeof(orc_plan));
    p->g = *g;
    p->Tw = orc_pulse_support(g);
    p->G = orc_effective_G(g);
    p->nq = g->Q * p->Tw + 1;
    p->gmax = orc_gamma_max(g);
    p->t0 = p->Tw / g->fs;
    p->tab = (double*)malloc(sizeof(double) * (size_t)p->G * p->nq);
    orc_pulse_table(g, p->tab, 1);
    long N = (long)g->img_w * g->img_h;
    if (!pix) npix = N;
    p->npix = npix;
    p->pix = (long*)malloc(sizeof(long) * (npix > 0 ? npix : 1));
    for (long s = 0; s < npix; ++s) p->pix[s] = pix ? pix[s] : s;
    int nall = g->n_tx * (1 + g->n_rx);
    double* all = (double*)malloc(sizeof(double) * nall);
    int n = 0;
    for (int i = 0; i < g->n_tx; ++i) all[n++] = g->tx_x[i];
    for (int i = 0; i < g->n_tx; ++i)
        for (int j = 0; j < g->n_rx; ++j) all[n++] = g->tx_x[i] + g->rx_offset[j];
    qsort(all, nall, sizeof(double), cmp_double);
    p->pos = (double*)malloc(sizeof(double) * (nall + g->n_tx));
    p->pos_tx = (int*)calloc(nall + g->n_tx, sizeof(int));
    p->npos = 0;
    for (int a = 0; a < nall; ++a)
        if (p->npos == 0 || all[a] != p->pos[p->npos - 1]) p->pos[p->npos++] = all[a];
    free(all);
    const int nshared = p->npos;
    p->tx_pos = (int*)malloc(sizeof(int) * g->n_tx);
    p->rx_pos = (int*)malloc(sizeof(int) * g->n_tx * g->n_rx);
    for (int i = 0; i < g->n_tx; ++i) {
        p->tx_pos[i] = find_pos(p->pos, nshared, g->tx_x[i]);
        for (int j = 0; j < g->n_rx; ++j)
            p->rx_pos[i * g->n_rx + j] = find_pos(p->pos, nshared, g->tx_x[i] + g->rx_offset[j]);
    }
    if (g->tilt != 0.0) {
        /* a tilted transmitter's legs weigh differently from a receiver's at the same place */
        for (int i = 0; i < g->n_tx; ++i) {
            p->pos[p->npos] = g->tx_x[i];
            p->pos_tx[p->npos] = 1;
            p->tx_pos[i] = p->npos++;
        }
    }
    p->tau_row = (double*)malloc(sizeof(double) * g->img_h);
    for (int r = 0; r < g->img_h; ++r)
        p->tau_row[r] = orc_transmission(g, g->z0 + (r + 0.5) * g->pitch);
    p->leg = (double**)calloc(p->npos, sizeof(double*));
    /* keep private copies of the transducer arrays */
    double* tx = (double*)malloc(sizeof(double) * g->n_tx);
    double* rx = (double*)malloc(sizeof(double) * g->n_rx);
    memcpy(tx, g->tx_x, sizeof(double) * g->n_tx);
    memcpy(rx, g->rx_offset, sizeof(double) * g->n_rx);
    p->g.tx_x = tx;
    p->g.rx_offset = rx;
    return p;
}

void orc_plan_destroy(orc_plan* p)
{
    if (!p) return;
    for (int a = 0; a < p->npos; ++a) free(p->leg[a]);
    free(p->leg);
    free(p->tab);
    free(p->pix);
    free(p->pos);
    free(p->pos_tx);
    free(p->tx_pos);
    free(p->rx_pos);
    free(p->tau_row);
    free((void*)p->g.tx_x);
    free((void*)p->g.rx_offset);
    free(p);
}

const double* orc_plan_table(const orc_plan* p) { return p->tab; }

/* legs (T, gamma, phi) from one transducer position to every plan pixel */
static void ensure_pos(orc_plan* p, int a, int nthreads)
{
    if (p->leg[a]) return;
    const orc_geom* g = &p->g;
    double* L = (double*)malloc(sizeof(double) * 3 * (p->npix > 0 ? p->npix : 1));
    double u = p->pos[a];
    #pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (long s = 0; s < p->npix; ++s) {
        long v = p->pix[s];
        int r = (int)(v / g->img_w), c = (int)(v % g->img_w);
        double xc = g->x0 + (c + 0.5) * g->pitch;
        double zr = g->z0 + (r + 0.5) * g->pitch;
        double T, gm, Th, th1;
        orc_leg(g, xc - u, zr, &T, &gm, &Th, &th1);
        /* eq. 12: the beam-profile angle is the sum of the layer angles (or the
         * first-layer angle); a tilted transmitter's beam axis is turned by
         * the firing angle toward +x, so the signed angle of the ray counts */
        double ang = g->apod_first ? th1 : Th;
        if (p->pos_tx[a]) ang = (xc - u >= 0.0 ? ang : -ang) - g->tilt;
        double cth = cos(ang);
        L[3 * s + 0] = T;
        L[3 * s + 1] = gm;
        L[3 * s + 2] = cth > 0.0 ? pow(cth, g->beta) : 0.0;   /* eq. 12 factor */
    }
    p->leg[a] = L;
}

static void pair_from_legs(const orc_plan* p, long s, int k, double* T, double* gamma, double* w)
{
    const orc_geom* g = &p->g;
    int i = k / g->n_rx;
    const double* lt = p->leg[p->tx_pos[i]] + 3 * s;
    const double* lr = p->leg[p->rx_pos[k]] + 3 * s;
    long v = p->pix[s];
    int r = (int)(v / g->img_w);
    *T = lt[0] + lr[0];
    *gamma = lt[1] + lr[1];
    *w = p->tau_row[r] * lt[2] * lr[2];
}

void orc_plan_pair(orc_plan* p, long s, int k, double* T, double* gamma, double* w)
{
    int i = k / p->g.n_rx;
    ensure_pos(p, p->tx_pos[i], 1);
    ensure_pos(p, p->rx_pos[k], 1);
    pair_from_legs(p, s, k, T, gamma, w);
}

/* bilinear read of the tabulated h~ (zero outside the open window 0 < tau < t0) */
double orc_plan_H(const orc_plan* p, double gamma, double tau)
{
    if (!(tau > 0.0 && tau < p->t0)) return 0.0;
    int last = p->nq - 1;
    double u = tau * p->g.fs * p->g.Q;
    int q = (int)floor(u);
    if (q > last - 1) q = last - 1;
    double phi = u - q;
    if (p->G == 1)
        return (1.0 - phi) * p->tab[q] + phi * p->tab[q + 1];
    double v = gamma / p->gmax * (p->G - 1);
    if (v < 0.0) v = 0.0;
    if (v > p->G - 1) v = p->G - 1;
    int gi = (int)floor(v);
    if (gi > p->G - 2) gi = p->G - 2;
    double psi = v - gi;
    const double* t0 = p->tab + (long)gi * p->nq;
    const double* t1 = t0 + p->nq;
    return (1.0 - psi) * ((1.0 - phi) * t0[q] + phi * t0[q + 1]) +
           psi * ((1.0 - phi) * t1[q] + phi * t1[q + 1]);
}

static void ensure_all_positions(orc_plan* p, int nthreads)
{
    for (int a = 0; a < p->npos; ++a) ensure_pos(p, a, nthreads);
}

/* taps of one pair: all n with 0 < n/fs - T < t0 inside the record */
static void tap_range(const orc_plan* p, double T, int* n_lo, int* n_hi)
{
    double fs = p->g.fs;
    long lo = (long)floor(T * fs);
    long hi = (long)ceil((T + p->t0) * fs);
    if (lo < 0) lo = 0;
    if (hi > p->g.n_samples - 1) hi = p->g.n_samples - 1;
    *n_lo = (int)lo;
    *n_hi = (int)hi;
}

/* y = A x restricted to A-scans [k_lo, k_hi) (eq. 13 summed over voxels) */
void orc_forward(orc_plan* p, const double* x, double* y, int k_lo, int k_hi, int nthreads)
{
    const orc_geom* g = &p->g;
    int M = g->n_samples;
    for (int k = k_lo; k < k_hi; ++k) {
        ensure_pos(p, p->tx_pos[k / g->n_rx], nthreads);
        ensure_pos(p, p->rx_pos[k], nthreads);
    }
    #pragma omp parallel for schedule(dynamic) num_threads(nthreads)
    for (int k = k_lo; k < k_hi; ++k) {
        double* yk = y + (long)(k - k_lo) * M;
        for (int n = 0; n < M; ++n) yk[n] = 0.0;
        for (long s = 0; s < p->npix; ++s) {
            double xv = x[p->pix[s]];
            if (xv == 0.0) continue;
            double T, gm, w;
            pair_from_legs(p, s, k, &T, &gm, &w);
            if (w == 0.0) continue;
            int n0, n1;
            tap_range(p, T, &n0, &n1);
            for (int n = n0; n <= n1; ++n)
                yk[n] += w * orc_plan_H(p, gm, n / g->fs - T) * xv;
        }
    }
}

/* b = A^T r for the plan's pixels */
void orc_backproject(orc_plan* p, const double* r, double* b, int nthreads)
{
    const orc_geom* g = &p->g;
    int M = g->n_samples, K = g->n_tx * g->n_rx;
    ensure_all_positions(p, nthreads);
    #pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (long s = 0; s < p->npix; ++s) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) {
            double T, gm, w;
            pair_from_legs(p, s, k, &T, &gm, &w);
            if (w == 0.0) continue;
            int n0, n1;
            tap_range(p, T, &n0, &n1);
            const double* rk = r + (long)k * M;
            for (int n = n0; n <= n1; ++n)
                acc += w * orc_plan_H(p, gm, n / g->fs - T) * rk[n];
        }
        b[s] = acc;
    }
}

/* dense (K*M) x N matrix, built column by column (tiny grids only) */
void orc_dense_A(orc_plan* p, double* A)
{
    const orc_geom* g = &p->g;
    int M = g->n_samples, K = g->n_tx * g->n_rx;
    long N = p->npix;
    ensure_all_positions(p, 1);
    memset(A, 0, sizeof(double) * (size_t)K * M * N);
    for (long s = 0; s < N; ++s)
        for (int k = 0; k < K; ++k) {
            double T, gm, w;
            pair_from_legs(p, s, k, &T, &gm, &w);
            for (int n = 0; n < M; ++n)
                A[((long)k * M + n) * N + s] = w * orc_plan_H(p, gm, n / g->fs - T);
        }
}

/* D of eq. 1: one column per receiver offset, the unattenuated pulse delayed
 * by the direct path |o_j| / c_1 along the array */
void orc_direct_columns(orc_plan* p, double* d)
{
    const orc_geom* g = &p->g;
    int M = g->n_samples;
    for (int j = 0; j < g->n_rx; ++j) {
        double T = fabs(g->rx_offset[j]) / g->speed[0];
        for (int n = 0; n < M; ++n) d[(long)j * M + n] = orc_plan_H(p, 0.0, n / g->fs - T);
    }
}

/* e = (I - D (D^T D)^-1 D^T) r per A-scan, gk = least-squares gains */
void orc_project(orc_plan* p, const double* r, double* e, double* gk)
{
    const orc_geom* g = &p->g;
    int M = g->n_samples, K = g->n_tx * g->n_rx;
    if (!g->direct_arrival) {
        memcpy(e, r, sizeof(double) * (size_t)K * M);
        if (gk) for (int k = 0; k < K; ++k) gk[k] = 0.0;
        return;
    }
    double* d = (double*)malloc(sizeof(double) * (size_t)g->n_rx * M);
    orc_direct_columns(p, d);
    for (int k = 0; k < K; ++k) {
        const double* dj = d + (long)(k % g->n_rx) * M;
        const double* rk = r + (long)k * M;
        double* ek = e + (long)k * M;
        double dd = 0.0, dr = 0.0;
        for (int n = 0; n < M; ++n) { dd += dj[n] * dj[n]; dr += dj[n] * rk[n]; }
        double gain = dd > 0.0 ? dr / dd : 0.0;
        for (int n = 0; n < M; ++n) ek[n] = rk[n] - gain * dj[n];
        if (gk) gk[k] = gain;
    }
    free(d);
}

/* ------------------------------------------------------------------ */
/* QGGMRF prior                                                        */
/* ------------------------------------------------------------------ */
double orc_rho(const orc_prior* pr, double delta, double sigma)
{
    double ad = fabs(delta);
    if (ad == 0.0) return 0.0;
    double u = pow(ad / (pr->T * sigma), pr->q - pr->p);
    return pow(ad, pr->p) / (pr->p * pow(sigma, pr->p)) * (u / (1.0 + u));   /* eq. 15 */
}

double orc_drho(const orc_prior* pr, double delta, double sigma)
{
    double ad = fabs(delta);
    if (ad == 0.0) return 0.0;
    double u = pow(ad / (pr->T * sigma), pr->q - pr->p);
    double sgn = delta > 0.0 ? 1.0 : -1.0;
    return sgn * pow(ad, pr->p - 1.0) / pow(sigma, pr->p) * (u / (1.0 + u)) *
           (1.0 + (pr->q - pr->p) / (pr->p * (1.0 + u)));
}

/* rho'(delta) / delta: curvature of the symmetric quadratic bound */
double orc_kappa(const orc_prior* pr, double delta, double sigma)
{
    double ad = fabs(delta);
    if (ad <= 1e-150 * pr->T * sigma)   /* limit delta -> 0 for q = 2 */
        return 2.0 / (pr->p * sigma * sigma * pow(pr->T, 2.0 - pr->p));
    return orc_drho(pr, delta, sigma) / delta;
}

static double row_weight(const orc_geom* g, const orc_prior* pr, int r)
{
    /* m_s of eq. 17: depth measured from the transducer plane */
    double z = g->z0 + (r + 0.5) * g->pitch;
    double zmax = g->z0 + (g->img_h - 0.5) * g->pitch;
    return 1.0 + (pr->m - 1.0) * pow(z / zmax, pr->a);
}

/* the four forward neighbours (E, SW, S, SE) enumerate each unordered
 * 8-neighbour clique once; weights 1 and 1/sqrt(2), normalised to sum 1 */
static const int NB_DR[4] = {0, 1, 1, 1};
static const int NB_DC[4] = {1, -1, 0, 1};

static double nb_weight(int t)
{
    double be = 1.0 / (4.0 + 4.0 / sqrt(2.0));
    return (t == 0 || t == 2) ? be : be / sqrt(2.0);
}

double orc_prior_cost(const orc_geom* g, const orc_prior* pr, const double* x)
{
    int W = g->img_w, H = g->img_h;
    double acc = 0.0;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c)
            for (int t = 0; t < 4; ++t) {
                int r2 = r + NB_DR[t], c2 = c + NB_DC[t];
                if (r2 < 0 || r2 >= H || c2 < 0 || c2 >= W) continue;
                double sg = pr->sigma0 * sqrt(row_weight(g, pr, r) * row_weight(g, pr, r2));  /* eq. 16 */
                acc += nb_weight(t) * orc_rho(pr, x[r * W + c] - x[r2 * W + c2], sg);
            }
    return acc;
}

void orc_prior_grad(const orc_geom* g, const orc_prior* pr, const double* x, double* grad)
{
    int W = g->img_w, H = g->img_h;
    for (long v = 0; v < (long)W * H; ++v) grad[v] = 0.0;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c)
            for (int t = 0; t < 4; ++t) {
                int r2 = r + NB_DR[t], c2 = c + NB_DC[t];
                if (r2 < 0 || r2 >= H || c2 < 0 || c2 >= W) continue;
                double sg = pr->sigma0 * sqrt(row_weight(g, pr, r) * row_weight(g, pr, r2));
                double dr = nb_weight(t) * orc_drho(pr, x[r * W + c] - x[r2 * W + c2], sg);
                grad[r * W + c] += dr;
                grad[r2 * W + c2] -= dr;
            }
}

double orc_prior_curv(const orc_geom* g, const orc_prior* pr, const double* x, const double* d)
{
    int W = g->img_w, H = g->img_h;
    double acc = 0.0;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c)
            for (int t = 0; t < 4; ++t) {
                int r2 = r + NB_DR[t], c2 = c + NB_DC[t];
                if (r2 < 0 || r2 >= H || c2 < 0 || c2 >= W) continue;
                double sg = pr->sigma0 * sqrt(row_weight(g, pr, r) * row_weight(g, pr, r2));
                double dd = d[r * W + c] - d[r2 * W + c2];
                acc += nb_weight(t) * orc_kappa(pr, x[r * W + c] - x[r2 * W + c2], sg) * dd * dd;
            }
    return acc;
}

/* ------------------------------------------------------------------ */
/* MAP iteration                                                       */
/* ------------------------------------------------------------------ */
int orc_reconstruct(orc_plan* p, const orc_prior* pr, const double* y, int n_iter,
                    double* x, int x_given, double* gk, double* cost, double* gnorm,
                    int nthreads)
{
    /* Fixed iteration (the paper optimises eq. 18 by ICD, which updates one
     * pixel at a time; this parallel form reaches the same unique minimiser):
     * Polak-Ribiere+ conjugate directions, each step the minimiser along d of
     * the exact data term plus the symmetric quadratic bound of the prior, so
     * the cost never increases.  A direction that is not a descent direction
     * is replaced by the negative gradient. */
    const orc_geom* g = &p->g;
    long N = (long)g->img_w * g->img_h;
    int K = g->n_tx * g->n_rx, M = g->n_samples;
    long KM = (long)K * M;
    if (p->npix != N) return -1;
    double s2 = pr->sigma_noise * pr->sigma_noise;
    double* r = (double*)malloc(sizeof(double) * KM);
    double* e = (double*)malloc(sizeof(double) * KM);
    double* q = (double*)malloc(sizeof(double) * KM);
    double* grad = (double*)malloc(sizeof(double) * N);
    double* gprev = (double*)calloc(N, sizeof(double));
    double* gr = (double*)malloc(sizeof(double) * N);
    double* d = (double*)calloc(N, sizeof(double));
    if (!x_given) for (long v = 0; v < N; ++v) x[v] = 0.0;
    /* residual of the data term, with the direct arrivals projected out */
    orc_forward(p, x, r, 0, K, nthreads);
    for (long a = 0; a < KM; ++a) r[a] = y[a] - r[a];
    orc_project(p, r, e, NULL);
    double gg_prev = 0.0;
    for (int it = 0; it < n_iter; ++it) {
        orc_backproject(p, e, grad, nthreads);               /* A^T e */
        orc_prior_grad(g, pr, x, gr);
        double gg = 0.0, ggp = 0.0;
        for (long v = 0; v < N; ++v) {
            grad[v] = -grad[v] / s2 + gr[v];                  /* gradient of eq. 18 */
            gg += grad[v] * grad[v];
            ggp += grad[v] * gprev[v];
        }
        if (gnorm) gnorm[it] = sqrt(gg);
        double beta = 0.0;
        if (it > 0 && gg_prev > 0.0) {
            beta = (gg - ggp) / gg_prev;
            if (beta < 0.0) beta = 0.0;
        }
        double gd = 0.0;
        for (long v = 0; v < N; ++v) {
            d[v] = -grad[v] + beta * d[v];
            gd += grad[v] * d[v];
        }
        if (!(gd < 0.0)) {
            gd = 0.0;
            for (long v = 0; v < N; ++v) { d[v] = -grad[v]; gd -= grad[v] * grad[v]; }
        }
        orc_forward(p, d, r, 0, K, nthreads);                 /* A d */
        orc_project(p, r, q, NULL);                           /* P A d */
        double qq = 0.0;
        for (long a = 0; a < KM; ++a) qq += q[a] * q[a];
        double den = qq / s2 + orc_prior_curv(g, pr, x, d);
        double alpha = den > 0.0 ? -gd / den : 0.0;
        for (long v = 0; v < N; ++v) x[v] += alpha * d[v];
        for (long a = 0; a < KM; ++a) e[a] -= alpha * q[a];
        for (long v = 0; v < N; ++v) gprev[v] = grad[v];
        gg_prev = gg;
        if (cost) {
            double ee = 0.0;
            for (long a = 0; a < KM; ++a) ee += e[a] * e[a];
            cost[it] = ee / (2.0 * s2) + orc_prior_cost(g, pr, x);
        }
    }
    if (gk) {
        orc_forward(p, x, r, 0, K, nthreads);
        for (long a = 0; a < KM; ++a) r[a] = y[a] - r[a];
        orc_project(p, r, q, gk);
    }
    free(r); free(e); free(q); free(grad); free(gprev); free(gr); free(d);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Iterative coordinate descent                                        */
/* ------------------------------------------------------------------ */
void orc_column_norms(orc_plan* p, double* out, int nthreads)
{
    const orc_geom* g = &p->g;
    int K = g->n_tx * g->n_rx;
    ensure_all_positions(p, nthreads);
    #pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (long s = 0; s < p->npix; ++s) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) {
            double T, gm, w;
            pair_from_legs(p, s, k, &T, &gm, &w);
            if (w == 0.0) continue;
            int n0, n1;
            tap_range(p, T, &n0, &n1);
            for (int n = n0; n <= n1; ++n) {
                double a = w * orc_plan_H(p, gm, n / g->fs - T);   /* entry (k, n) of column s */
                acc += a * a;
            }
        }
        out[s] = acc;
    }
}

int orc_icd(orc_plan* p, const orc_prior* pr, const double* y, int n_sweeps, int spacing,
            double* x, int x_given, double* gk, double* cost, int nthreads)
{
    /* ICD on the cost of eq. 18 with g eliminated (e = P (y - A x)).  For pixel
     * v the data term along x_v is the quadratic theta1 u + theta2 u^2 / 2 with
     * theta1 = -(A^T e)_v / sigma^2 and theta2 = |A_v|^2 / sigma^2 (the column
     * before the projection: an upper bound of the projected curvature), and
     * each clique {v, r} is replaced by its symmetric quadratic bound with
     * curvature b kappa(x_v - x_r).  The 1-D minimiser of that surrogate is
     *     dx_v = -(theta1 + sum_r b rho'(x_v - x_r)) / (theta2 + sum_r b kappa).
     * Pixels of one colour share no clique; the group moves along dx by the
     * step alpha that minimises the exact data term plus the prior bound on
     * that line (alpha = 1 for a group of one pixel). */
    const orc_geom* g = &p->g;
    int W = g->img_w, H = g->img_h;
    long N = (long)W * H;
    int K = g->n_tx * g->n_rx, M = g->n_samples;
    long KM = (long)K * M;
    if (p->npix != N) return -1;
    if (spacing < 2) return -2;
    double s2 = pr->sigma_noise * pr->sigma_noise;
    double* cn = (double*)malloc(sizeof(double) * N);
    double* b = (double*)malloc(sizeof(double) * N);
    double* dx = (double*)calloc(N, sizeof(double));
    double* r = (double*)malloc(sizeof(double) * KM);
    double* e = (double*)malloc(sizeof(double) * KM);
    double* q = (double*)malloc(sizeof(double) * KM);
    orc_column_norms(p, cn, nthreads);
    if (!x_given) for (long v = 0; v < N; ++v) x[v] = 0.0;
    orc_forward(p, x, r, 0, K, nthreads);
    for (long a = 0; a < KM; ++a) r[a] = y[a] - r[a];
    orc_project(p, r, e, NULL);
    for (int sw = 0; sw < n_sweeps; ++sw) {
        for (int colour = 0; colour < spacing * spacing; ++colour) {
            int cr = colour / spacing, cc = colour % spacing;
            if (cr >= H || cc >= W) continue;
            orc_backproject(p, e, b, nthreads);                  /* A^T e */
            double gd = 0.0, curv = 0.0;
            for (int rr = cr; rr < H; rr += spacing)
                for (int c = cc; c < W; c += spacing) {
                    long v = (long)rr * W + c;
                    double gR = 0.0, D = 0.0;
                    for (int dr = -1; dr <= 1; ++dr)
                        for (int dc = -1; dc <= 1; ++dc) {
                            if (dr == 0 && dc == 0) continue;
                            int r2 = rr + dr, c2 = c + dc;
                            if (r2 < 0 || r2 >= H || c2 < 0 || c2 >= W) continue;
                            double sg = pr->sigma0 * sqrt(row_weight(g, pr, rr) * row_weight(g, pr, r2));
                            double wgt = nb_weight(dr == 0 || dc == 0 ? 0 : 1);
                            double delta = x[v] - x[(long)r2 * W + c2];
                            gR += wgt * orc_drho(pr, delta, sg);
                            D += wgt * orc_kappa(pr, delta, sg);
                        }
                    double grad = -b[v] / s2 + gR;
                    double den = cn[v] / s2 + D;
                    dx[v] = den > 0.0 ? -grad / den : 0.0;
                    gd += grad * dx[v];
                    curv += D * dx[v] * dx[v];
                }
            orc_forward(p, dx, r, 0, K, nthreads);               /* A dx */
            orc_project(p, r, q, NULL);
            double qq = 0.0;
            for (long a = 0; a < KM; ++a) qq += q[a] * q[a];
            double den = qq / s2 + curv;
            double alpha = den > 0.0 ? -gd / den : 0.0;
            for (int rr = cr; rr < H; rr += spacing)
                for (int c = cc; c < W; c += spacing) {
                    long v = (long)rr * W + c;
                    x[v] += alpha * dx[v];
                    dx[v] = 0.0;
                }
            for (long a = 0; a < KM; ++a) e[a] -= alpha * q[a];
        }
        if (cost) {
            double ee = 0.0;
            for (long a = 0; a < KM; ++a) ee += e[a] * e[a];
            cost[sw] = ee / (2.0 * s2) + orc_prior_cost(g, pr, x);
        }
    }
    if (gk) {
        orc_forward(p, x, r, 0, K, nthreads);
        for (long a = 0; a < KM; ++a) r[a] = y[a] - r[a];
        orc_project(p, r, q, gk);
    }
    free(cn); free(b); free(dx); free(r); free(e); free(q);
    return 0;
}
