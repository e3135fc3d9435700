/*
 * FP64 CPU oracle for multi-layer collimated-beam MBIR (Alanazi et al.,
 * "Model-Based Reconstruction for Collimated Beam Ultrasound Systems").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * restatement of the paper's model used to check the CUDA library.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it; the product path never calls it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Every quantity is double precision.  Units are SI (m, s, m/s, kg/m^3);
 * attenuation is given in s/m (Np per Hz per metre) as in Section 2, eq. 3.
 * Pixel v = r * img_w + c, row r is depth, column c is lateral.
 * A-scan k = i * n_rx + j (Tx position i, receiver j).
 */
#ifndef MBIR_ORACLE_H
#define MBIR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LAYERS 8

typedef struct {
    int n_layers;
    double thickness[ORC_MAX_LAYERS];  /* m; the last layer extends downwards */
    double speed[ORC_MAX_LAYERS];      /* m/s */
    double atten[ORC_MAX_LAYERS];      /* s/m (alpha of eq. 3) */
    double density[ORC_MAX_LAYERS];    /* kg/m^3 */
    int img_w, img_h;
    double pitch, x0, z0;              /* pixel (r,c) centre: x0+(c+.5)pitch, z0+(r+.5)pitch */
    int n_tx;
    const double* tx_x;                /* Tx lateral positions (depth 0) */
    int n_rx;
    const double* rx_offset;           /* receiver offsets from the Tx position */
    double fs;                         /* sampling rate, Hz */
    int n_samples;                     /* M */
    double fc, n_cycles;               /* Gaussian-modulated cosine pulse */
    double beta;                       /* apodization power, eq. 12 */
    int direct_arrival;                /* 1: model D g of eq. 1 */
    double gamma_max;                  /* s; <= 0 selects the default rule */
    int G, Q;                          /* pulse-table gamma bins and phases per sample */
    double tilt;                       /* transmitter firing angle (rad) toward +x (Section 3: 5 degrees) */
    int apod_first;                    /* 1: eq. 12 with the first-layer angle instead of the angle sum */
} orc_geom;

typedef struct {
    double p, q, T, sigma0, m, a;      /* QGGMRF, eq. 15-17 */
    double sigma_noise;                /* sigma of eq. 2 */
} orc_prior;

typedef struct orc_plan orc_plan;

/* pulse (Section 2, eq. 9-10) */
int    orc_pulse_support(const orc_geom* g);            /* T_w in samples */
double orc_pulse(const orc_geom* g, double t);          /* s(t) */
double orc_gamma_max(const orc_geom* g);
int    orc_effective_G(const orc_geom* g);
void   orc_pulse_table(const orc_geom* g, double* tab, int panels_scale); /* G x (Q*Tw+1) */

/* one leg, eq. 4-6 */
void orc_leg(const orc_geom* g, double h, double z,
             double* T, double* gamma, double* Theta, double* theta1);
double orc_transmission(const orc_geom* g, double z);

/* plans: leg cache over a pixel subset (NULL = all pixels) */
orc_plan* orc_plan_create(const orc_geom* g, const long* pix, long npix, int nthreads);
void      orc_plan_destroy(orc_plan* p);
const double* orc_plan_table(const orc_plan* p);
void   orc_plan_pair(orc_plan* p, long slot, int k, double* T, double* gamma, double* w);
double orc_plan_H(const orc_plan* p, double gamma, double tau);

/* operators (eq. 11, 13 and the adjoint) */
void orc_forward(orc_plan* p, const double* x, double* y, int k_lo, int k_hi, int nthreads);
void orc_backproject(orc_plan* p, const double* r, double* b, int nthreads);
void orc_dense_A(orc_plan* p, double* A);
void orc_direct_columns(orc_plan* p, double* d);      /* n_rx x M */
void orc_project(orc_plan* p, const double* r, double* e, double* gk);

/* prior (eq. 14-17) */
double orc_prior_cost(const orc_geom* g, const orc_prior* pr, const double* x);
void   orc_prior_grad(const orc_geom* g, const orc_prior* pr, const double* x, double* grad);
double orc_prior_curv(const orc_geom* g, const orc_prior* pr, const double* x, const double* d);
double orc_rho(const orc_prior* pr, double delta, double sigma);
double orc_drho(const orc_prior* pr, double delta, double sigma);
double orc_kappa(const orc_prior* pr, double delta, double sigma);

/* MAP estimate of eq. 18 by the fixed majorize-minimize conjugate-gradient iteration */
int orc_reconstruct(orc_plan* p, const orc_prior* pr, const double* y, int n_iter,
                    double* x, int x_given, double* gk, double* cost, double* gnorm,
                    int nthreads);

/* ||A_v||^2 per plan pixel: the sum over A-scans and taps of (w H)^2 */
void orc_column_norms(orc_plan* p, double* out, int nthreads);

/* MAP estimate of eq. 18 by coloured iterative coordinate descent (the
 * paper's optimiser, Section 2 "Optimization"): pixels (r, c) are grouped by
 * (r mod spacing, c mod spacing); each group takes every member's 1-D ICD
 * update at once, scaled by one majorize-minimize step.  A group of one pixel
 * is the sequential ICD update exactly.  cost[sweep] after every sweep.
 * Returns -1 unless the plan covers every pixel, -2 for spacing < 2. */
int orc_icd(orc_plan* p, const orc_prior* pr, const double* y, int n_sweeps, int spacing,
            double* x, int x_given, double* gk, double* cost, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
