/*
 * mbir.h - C ABI of the GB300 multi-layer collimated-beam MBIR library.
 *
 * The library applies the physics-based forward model A of Alanazi et al.,
 * "Model-Based Reconstruction for Collimated Beam Ultrasound Systems"
 * (Section 2, eq. 1-13), its adjoint, the direct-arrival term of eq. 1 and the
 * QGGMRF prior of eq. 14-17, and minimises the MAP cost of eq. 18, all in
 * hand-written CUDA kernels for sm_103a.
 *
 * Conventions
 *   - SI units (m, s, m/s, kg/m^3).  Attenuation alpha is given in
 *     Np / (MHz m) (the paper's "/Hz m" read with f in MHz, Section 3).
 *   - Image pixel v = r * img_w + c; row r is depth, column c is lateral.
 *     Pixel centre: (img_x0_m + (c + 0.5) pitch_m, img_z0_m + (r + 0.5) pitch_m).
 *     Transducers sit at depth 0 in layer 1.
 *   - A-scan k = i * n_rx + j: transmitter position i (lateral tx_x_m[i]),
 *     receiver j (lateral tx_x_m[i] + rx_offset_m[j]).  y is K x M row-major,
 *     K = n_tx * n_rx, M = n_samples, sample n at time n / fs_hz.
 *   - Device pointers are owned by the caller (e.g. a torch tensor's
 *     data_ptr) and must stay valid until the stream reaches the call.  All
 *     device work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and is asynchronous unless stated otherwise.
 *   - Every call returns MBIR_OK (0) or a negative MBIR_ERR_* code; outputs
 *     are untouched on an argument error.  mbir_error_string gives the text.
 *   - A geometry handle may be used from one host thread at a time; calls
 *     that share a handle must be ordered on one stream (the handle owns the
 *     reconstruction workspace).
 */
#ifndef MBIR_H
#define MBIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MBIR_OK               0
#define MBIR_ERR_INVALID_ARG (-1)  /* bad size, pointer, layer or prior value */
#define MBIR_ERR_OOM         (-2)  /* device or host allocation failed */
#define MBIR_ERR_CUDA        (-3)  /* a CUDA runtime call or launch failed */
#define MBIR_ERR_NONFINITE   (-4)  /* the data or an iterate is NaN/Inf */
#define MBIR_ERR_TIMEOUT     (-5)  /* a bounded wait gave up */
#define MBIR_ERR_BUSY        (-6)  /* admission refused: over the memory budget */
#define MBIR_ERR_UNSUPPORTED (-7)  /* option not available for this geometry */
#define MBIR_ERR_CANCELLED   (-8)  /* a request was cancelled */
#define MBIR_ERR_NOT_READY   (-9)  /* a request has not finished yet */

#define MBIR_MAX_LAYERS 8

typedef enum {
    MBIR_PREC_FP32 = 0,          /* y, residual and pulse table in FP32 */
    MBIR_PREC_BF16 = 1           /* y / residual copy and pulse table stored BF16, FP32 math */
} mbir_precision;

typedef enum {
    MBIR_MODE_AUTO = 0,          /* TAB when the leg table fits, else OTF */
    MBIR_MODE_OTF = 1,           /* travel times solved in registers on every apply */
    MBIR_MODE_TAB = 2            /* legs solved once per geometry, kept in device memory */
} mbir_mode;

/* Angle of eq. 12's beam profile cos^beta(angle).  ANGLE_SUM follows eq. 12
 * (the sum of the layer angles); FIRST_ANGLE is a variant that uses the
 * first-layer angle only. */
typedef enum {
    MBIR_APOD_ANGLE_SUM = 0,
    MBIR_APOD_FIRST_ANGLE = 1
} mbir_apodization;

/*
 * Geometry of one scan (Section 2 "Multi-layered structures", eq. 3-6, and the
 * acquisition of Section 3).  Arrays are host memory and are copied.
 *   thickness_m[l], speed_mps[l], atten_np_per_mhz_m[l], density_kgm3[l]:
 *       layer l from the transducer plane down; the last layer extends below
 *       its thickness.  Density only enters the interface transmittance tau.
 *   pulse: Gaussian-modulated cosine at fc_hz whose envelope FWHM spans
 *       n_cycles periods; its window t0 (eq. 10) is ceil(8 sigma fs) samples.
 *   beta: apodization power of eq. 12.
 *   direct_arrival: 1 adds one direct-arrival column per A-scan (eq. 1).
 *   gamma_max_s: top of the pulse table's attenuation axis (s); 0 selects
 *       4 * sum_l alpha_l eta_l down to the deepest pixel centre.
 *   gamma_bins (G), phases (Q): pulse table of G attenuation bins and Q
 *       phases per sample, read by bilinear interpolation (0 selects 16, 16).
 *   flags: MBIR_FLAG_* below (0 for the defaults).
 *   firing_angle_rad: the transmitter's beam axis is turned by this angle
 *       toward +x (the Section 3 source is tilted by 5 degrees), so its
 *       factor of eq. 12 is cos^beta(signed ray angle - firing angle); the
 *       receivers are not tilted.  |angle| < pi/2; a nonzero angle needs TAB
 *       mode (MBIR_ERR_UNSUPPORTED with MBIR_MODE_OTF).
 *   apodization: mbir_apodization (0 selects eq. 12 as written).
 */
typedef struct {
    int n_layers;
    double thickness_m[MBIR_MAX_LAYERS];
    double speed_mps[MBIR_MAX_LAYERS];
    double atten_np_per_mhz_m[MBIR_MAX_LAYERS];
    double density_kgm3[MBIR_MAX_LAYERS];
    int img_w, img_h;
    double pitch_m, img_x0_m, img_z0_m;
    int n_tx;
    const double* tx_x_m;
    int n_rx;
    const double* rx_offset_m;
    double fs_hz;
    int n_samples;
    double fc_hz, n_cycles;
    double beta;
    int direct_arrival;
    double gamma_max_s;
    int gamma_bins, phases;
    int precision;               /* mbir_precision */
    int mode;                    /* mbir_mode */
    int flags;                   /* MBIR_FLAG_* */
    double firing_angle_rad;     /* transmitter beam axis turned toward +x (Section 3: 5 degrees); TAB mode */
    int apodization;             /* mbir_apodization */
} mbir_geometry_desc;

/* TAB mode normally also stores every A-scan's active pairs as records
 * grouped by first tap sample (the system matrix of Section 3) so that A x
 * and A^T stream them: 24 bytes per active pair for the CUDA-core kernels,
 * packed to 16 (FP32 form) or 12 bytes (BF16 form) for the tensor-core ones;
 * this flag keeps the on-the-fly record path of A x instead (less memory,
 * slower). */
#define MBIR_FLAG_NO_RECORDS 1

/* With records, A and A^T normally run on the tensor cores (both storage
 * forms).  Every tap of a pair shares one table phase (eq. 13 with the
 * bilinear table), so per A-scan and tile of 128 first-tap samples n0:
 *   A x: the pairs' weights times x are summed per (n0, table row), the sums
 *        multiplied by the table on the tensor cores and added along the
 *        product's anti-diagonals;
 *   A^T: the correlation of the residual with the table rows is one matrix
 *        product, and each pair combines four of its values into one
 *        contribution, which is rounded to a 64-bit fixed-point grid (one
 *        power-of-two scale per call, from max |e| and bounds of the weights
 *        and the table) and added to its pixel's integer sum; the exact sum is
 *        rounded once to FP32 (a non-finite residual gives NaN).
 * FP32 form: operands scaled by powers of two and split into two FP16 parts
 * (three products, FP32 accuracy); BF16 form: the stored BF16 residual and
 * table, the A x sums rounded once to BF16.  FP32 accumulation otherwise;
 * outputs are bitwise reproducible.  This flag keeps the CUDA-core kernels. */
#define MBIR_FLAG_NO_TENSOR_CORES 2

/* QGGMRF prior (eq. 15-17) and the noise sigma of eq. 2.
 * Requires 1 < p < q = 2 (Section 2, "Prior model"), T > 0, sigma0 > 0,
 * m > 0, a >= 0 and sigma_noise > 0. */
typedef struct {
    double p, q, T, sigma0, m, a;
    double sigma_noise;
} mbir_prior;

/* Per-call statistics (host memory).  cost may be NULL; when given it
 * receives min(cost_len, n_iter) values of the eq. 18 cost after each
 * iteration (this adds one device-to-host read per iteration). */
typedef struct {
    double* cost;
    int cost_len;
    int iterations;
    double grad_norm_first;
    double grad_norm_last;
} mbir_stats;

typedef struct {
    int64_t n_pixels, n_ascans, n_samples;
    int pulse_support;           /* T_w samples */
    int gamma_bins, phases;
    double gamma_max_s;
    int mode;                    /* resolved mbir_mode (OTF or TAB) */
    int precision;
    int64_t device_bytes;        /* tables + workspace held by the handle */
    int forward_window_spans;    /* sorted TAB records (CUDA-core A x): 32-sample spans per work unit, else 0 */
    double forward_window_ms[3]; /* CUDA-core A x times for windows of 1, 2 and 4 spans, measured at creation
                                  * when that kernel is the geometry's A x (0 otherwise) */
    int adjoint_groups;          /* transmitter groups of the CUDA-core A^T r work items */
    int adjoint_tensor_cores;    /* 1 if A^T runs on the tensor cores (see MBIR_FLAG_NO_TENSOR_CORES) */
    int forward_tensor_cores;    /* 1 if A x runs on the tensor cores */
    int64_t n_records;           /* TAB records: active (pixel, A-scan) pairs held, else 0 */
    int64_t record_bytes;        /* bytes of the record list as held: 24 per pair sorted (CUDA-core A x),
                                  * 16 (FP32 form) or 12 (BF16 form) packed for the tensor cores */
    int tc_forward_variant;      /* tensor-core A x variant in use: 0 record loads through the L1, 1 records
                                  * past the L1 and the gathered image kept there */
    int tc_adjoint_variant;      /* tensor-core A^T variant in use: 0 four, 1 six records per thread and batch */
    double tc_variant_ms[4];     /* their times measured at creation (A x 0, 1, A^T 0, 1; 0 if not timed):
                                  * each pool runs the faster of its two */
} mbir_geometry_info;

typedef struct mbir_geometry mbir_geometry;

/* Validate `d`, build the pulse table (eq. 9-10) on the host in FP64, copy
 * the layer, transducer and table data to the current device, and (TAB mode)
 * solve every leg once (the paper's "compute only once", Section 3).
 * Errors: MBIR_ERR_INVALID_ARG (n_layers outside 1..8, non-positive
 * thickness, speed, density, pitch, fs, fc, n_cycles, beta < 0, negative
 * attenuation, img_z0_m < 0, sizes < 1, NULL arrays, K*M or N above 2^31,
 * K above 65535),
 * MBIR_ERR_OOM, MBIR_ERR_CUDA, MBIR_ERR_UNSUPPORTED (the pulse table and two
 * padded residual rows exceed shared memory: with the default 16 x 16 FP32
 * table about 11,000 samples per A-scan, twice that in BF16).  *out is
 * untouched on error.  Synchronises `stream` before returning. */
int mbir_create_geometry(const mbir_geometry_desc* d, void* stream, mbir_geometry** out);

/* Free the handle and its device memory.  Accepts NULL.  The caller must
 * have finished every call that uses the handle. */
int mbir_destroy_geometry(mbir_geometry* g);

/* Bytes of device memory held by the handle (tables and workspace). */
size_t mbir_geometry_bytes(const mbir_geometry* g);

int mbir_geometry_get_info(const mbir_geometry* g, mbir_geometry_info* info);

/* Override the window of the CUDA-core A x (TAB records only): every warp of
 * that kernel then covers `spans` consecutive 32-sample spans (1, 2 or 4).
 * A tuning control with no counterpart in the paper; the output bits do not
 * depend on it.  Synchronises the device; the handle must not be in use by
 * another call or an engine.  Errors: MBIR_ERR_INVALID_ARG (other values),
 * MBIR_ERR_UNSUPPORTED (no sorted record list: OTF mode, or a geometry whose
 * A x runs on the tensor cores, which keeps only the packed records),
 * MBIR_ERR_OOM, MBIR_ERR_CUDA. */
int mbir_set_forward_window(mbir_geometry* g, int spans);

/* Override the variants of the tensor-core A x and A^T that the geometry
 * chose by timing at creation (see mbir_geometry_info): 0 or 1 each, -1
 * keeps the current one.  A tuning control with no counterpart in the paper;
 * the output bits do not depend on it.  The handle must not be in use by
 * another call or an engine (an engine reads the variants when a request is
 * admitted).  Errors: MBIR_ERR_INVALID_ARG (other values), MBIR_ERR_UNSUPPORTED
 * (a variant given for an apply that does not run on the tensor cores). */
int mbir_set_tensor_core_variants(mbir_geometry* g, int forward_variant, int adjoint_variant);

/* y = A x (eq. 11-13 summed over voxels).  x_dev: N floats.  y_dev: K x M,
 * float (FP32) or bfloat16 (BF16 precision).  Every output sample is written
 * (no accumulation into y). */
int mbir_forward(const mbir_geometry* g, const float* x_dev, void* y_dev, void* stream);

/* x = A^T r (adjoint of eq. 13).  r_dev: K x M, float (FP32) or bfloat16
 * (BF16 precision).  x_dev: N floats, overwritten. */
int mbir_backproject(const mbir_geometry* g, const void* r_dev, float* x_dev, void* stream);

/* x = A^T r like mbir_backproject, but without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate at the point of the call - real-time loops that forbid
 * allocator calls after start-up (an allocation can block for an unbounded
 * time), and processes whose device memory is one pool sized and handed out
 * in advance by another component.  (mbir_backproject may allocate its workspace on first use.)
 * Its scratch (the padded residual rows, K x (M + pulse support + pad)
 * floats, and one partial image per transmitter group) lives in one fixed
 * 16 MiB array inside the library, held by every GPU that loads the library
 * until the process exits.
 *   - Geometries whose scratch would exceed 16 MiB (for a 256 x 512 image,
 *     more than about 3 M residual samples) and BF16-precision geometries
 *     return MBIR_ERR_UNSUPPORTED.
 *   - Set-up is part of mbir_create_geometry: creating a geometry that this
 *     entry point takes looks up the array's device address on that device
 *     (once per device; where modules load lazily this is when the array's
 *     16 MiB are reserved) and loads the kernels of the call, so the call
 *     itself loads and allocates nothing.  The geometry's device must be
 *     current.
 *   - Every call rewrites the scratch before reading it, so no clearing is
 *     needed, but all calls share the one array: calls whose work overlaps on
 *     the GPU (other streams, other host threads) race and must be
 *     serialised by the caller.  The call also uses the geometry's adjoint
 *     work counter, so it must not overlap any other call that applies A^T
 *     with the same geometry (mbir_backproject, the reconstructions, an
 *     engine running a request of that geometry).
 * r_dev: K x M floats; x_dev: N floats, overwritten.  Asynchronous on
 * `stream`; no device memory is allocated or freed. */
int mbir_backproject_noalloc(const mbir_geometry* g, const float* r_dev, float* x_dev, void* stream);

/* Direct-arrival projection (eq. 1): per A-scan k, g_k = <d_k, r_k>/|d_k|^2
 * and e_k = r_k - g_k d_k, with d_k the unattenuated pulse delayed by
 * |rx_offset_m[j]| / speed_mps[0].  r_dev, e_dev: K x M floats (may alias);
 * gk_dev: K floats or NULL.  Without direct arrivals e = r and g = 0. */
int mbir_project(const mbir_geometry* g, const float* r_dev, float* e_dev, float* gk_dev,
                 void* stream);

/* y += D g (eq. 1): adds g_k times the direct-arrival column of A-scan k to
 * every A-scan.  gk_dev: K floats; y_dev: K x M floats, updated in place. */
int mbir_add_direct(const mbir_geometry* g, const float* gk_dev, float* y_dev, void* stream);

/* Gradient of the prior of eq. 14-17 at x: out_s = sum_r b_sr rho'(x_s - x_r).
 * x_dev, out_dev: N floats. */
int mbir_prior_gradient(const mbir_geometry* g, const mbir_prior* pr, const float* x_dev,
                        float* out_dev, void* stream);

/* MAP estimate of eq. 18.  y_dev: K x M (float, or bfloat16 in BF16
 * precision).  x_dev: N floats, the start when x_given != 0 (else zeros), the
 * estimate on return.  g_dev: K floats (direct-arrival gains) or NULL.
 * Iteration: Polak-Ribiere+ conjugate directions with the majorize-minimize
 * step of the exact data term plus the symmetric quadratic bound of the prior.
 * Synchronises `stream` before returning (it reads the convergence scalars).
 * Errors: MBIR_ERR_INVALID_ARG (prior outside 1 < p < q = 2 and friends,
 * n_iter < 0), MBIR_ERR_NONFINITE (the data or cost is NaN/Inf), MBIR_ERR_CUDA. */
int mbir_reconstruct(const mbir_geometry* g, const void* y_dev, const mbir_prior* pr,
                     int n_iter, float* x_dev, int x_given, float* g_dev, mbir_stats* st,
                     void* stream);

/* MAP estimate of eq. 18 by coloured iterative coordinate descent (Section 2
 * "Optimization": the paper optimises with ICD).  Pixels (r, c) are grouped
 * by colour (r mod spacing, c mod spacing); spacing >= 2 keeps the two ends
 * of every 8-neighbour clique in different colours.  For a colour, every
 * member v takes its 1-D ICD update
 *     dx_v = -(theta1 + sum_r b rho'(x_v - x_r)) / (theta2 + sum_r b kappa),
 * theta1 = -(A^T e)_v / sigma^2, theta2 = |A_v|^2 / sigma^2 (e the projected
 * residual; kappa = rho'/delta, the symmetric quadratic bound of each clique),
 * and the colour moves along dx by the step alpha that minimises the exact
 * data term plus the bound on that line; for a colour of one pixel
 * (spacing >= both image sides) alpha = 1 and this is sequential ICD in
 * raster order.  A sweep visits the spacing^2 colours in order (empty ones
 * skipped), each with A^T on the colour's pixels only, A of its update and
 * the projection; with TAB records and spacing <= 64 the A reads only the
 * colour's records (a per-colour copy of the record list, built on the first
 * call with that spacing and kept by g, as are the column norms, N floats).
 * Arguments as mbir_reconstruct, with n_sweeps in place of n_iter;
 * st->cost receives the cost after each sweep and the gradient norms are 0.
 * Synchronises `stream`.  Errors: as mbir_reconstruct, and
 * MBIR_ERR_INVALID_ARG for spacing outside 2..256. */
int mbir_reconstruct_icd(const mbir_geometry* g, const void* y_dev, const mbir_prior* pr,
                         int n_sweeps, int spacing, float* x_dev, int x_given, float* g_dev,
                         mbir_stats* st, void* stream);

/* |A_v|^2 per pixel (the coordinate descent's data curvature times sigma^2):
 * the sum over A-scans and taps inside the record of (w H)^2 with the FP32
 * pulse table.  out_dev: N floats.  Asynchronous on `stream`. */
int mbir_column_norms(const mbir_geometry* g, float* out_dev, void* stream);

/* mbir_reconstruct on host buffers: copies y_host (K x M float) in, runs, and
 * copies x_host (N floats) and g_host (K floats, may be NULL) out, all on
 * `stream`.  Synchronises the stream. */
int mbir_reconstruct_host(const mbir_geometry* g, const float* y_host, const mbir_prior* pr,
                          int n_iter, float* x_host, float* g_host, mbir_stats* st,
                          void* stream);

/*
 * Batched and served reconstructions (continuous batching).
 *
 * An engine advances many independent MAP problems (eq. 18) of uneven size
 * together, one iteration per step; each step is one launch of a captured
 * CUDA graph of grouped kernels over every active request.  Requests enter
 * and leave between steps: a queued request is admitted when its device
 * state fits the engine's byte budget, and retires after its own n_iter
 * iterations.  A request's result does not depend on which other requests
 * share its steps.  Geometries must be TAB mode with records (the default for
 * grid-aligned transducers); all active requests of one engine share one
 * precision.  An engine and its requests belong to the device current at
 * creation and are driven from one host thread and one stream.
 */
typedef struct mbir_engine mbir_engine;

/* budget_bytes: cap on the device state of admitted requests (their
 * geometries are owned by the caller and not counted); max_active: cap on
 * requests per step.  Errors: MBIR_ERR_INVALID_ARG, MBIR_ERR_CUDA. */
int mbir_engine_create(size_t budget_bytes, int max_active, mbir_engine** out);

/* Waits for the device, frees every request's state and the engine. */
int mbir_engine_destroy(mbir_engine* e);

/* Queues one reconstruction of y_dev (K x M, float or bfloat16 per the
 * geometry's precision; must stay valid until the request is done) with
 * prior `pr` and n_iter iterations.  x_dev (N floats) is the iterate, written
 * in place from zero; g_dev (K floats, may be NULL) receives the
 * direct-arrival gains at the end.  *ticket identifies the request.
 * Errors: MBIR_ERR_INVALID_ARG, MBIR_ERR_UNSUPPORTED (geometry not TAB with
 * records, table or record length beyond the engine's limits, other device),
 * MBIR_ERR_BUSY (the request alone exceeds the budget). */
int mbir_engine_submit(mbir_engine* e, const mbir_geometry* g, const void* y_dev, const mbir_prior* pr, int n_iter,
                       float* x_dev, float* g_dev, int64_t* ticket);

/* One engine step on `stream`: retire requests that finished, admit queued
 * requests that fit the budget (arrival order), then one MAP iteration of
 * every active request.  Asynchronous except for retirement, which reads each
 * finishing request's status.  *n_active / *n_queued (may be NULL) report the
 * engine's load after admission. */
int mbir_engine_step(mbir_engine* e, void* stream, int* n_active, int* n_queued);

/* *state: 0 queued, 1 running, 3 done; a negative MBIR_ERR_* if the request
 * failed (also returned). */
int mbir_engine_poll(mbir_engine* e, int64_t ticket, int* state);

/* Steps the engine until the request is done; MBIR_ERR_TIMEOUT if timeout_ms
 * of host time pass first (the request keeps running). */
int mbir_engine_wait(mbir_engine* e, int64_t ticket, int timeout_ms, void* stream);

/* Removes a queued or running request (state becomes MBIR_ERR_CANCELLED). */
int mbir_engine_cancel(mbir_engine* e, int64_t ticket, void* stream);

/* Device bytes of request state currently admitted. */
size_t mbir_engine_bytes_in_use(const mbir_engine* e);

/* Diagnostics for parity tests: per requested (pixel, A-scan) pair, the
 * device's travel time in samples (double, from its compensated FP32 pair),
 * total attenuation gamma (s) and weight w = tau * phi (eq. 12).
 * pix_host, k_host: n ints (host).  Outputs: n values each (host). */
int mbir_pair_quantities(const mbir_geometry* g, const int32_t* pix_host, const int32_t* k_host,
                         int n, double* T_samples_host, float* gamma_host, float* w_host);

/* Copy the pulse table used by the kernels (G x (Q*T_w + 1) doubles,
 * as built on the host) to host memory. */
int mbir_pulse_table(const mbir_geometry* g, double* out_host, size_t n);

/* Per-kernel device time of the A x and A^T r launches made inside
 * mbir_reconstruct while profiling is on (CUDA events on the call's stream,
 * read when the call synchronises).  Enabling adds two event records per
 * launch; it does not change results. */
typedef struct {
    int64_t forward_launches, backproject_launches;
    double forward_ms, backproject_ms;
} mbir_kernel_times;

int mbir_set_profiling(mbir_geometry* g, int enable);
int mbir_get_kernel_times(mbir_geometry* g, mbir_kernel_times* t, int reset);

/* Algorithmic work of one apply of A (or A^T): the number of (pixel, A-scan)
 * pairs with a non-zero weight and a tap inside the record, and the number of
 * taps (samples n with 0 < n - T < t0, n < M) over those pairs.  Computed on
 * the device from the geometry alone; synchronises the legacy stream. */
int mbir_count_taps(const mbir_geometry* g, int64_t* active_pairs, int64_t* taps);

/* Failure-detection self-test: launches a kernel whose bounded wait can never
 * be satisfied (an mbarrier that no arrival completes) and returns
 * MBIR_ERR_TIMEOUT once the wait gives up after max_cycles SM clocks
 * (1 .. 4e9), leaving the context usable.  The apply kernels use the same
 * bounded waits for their bulk copies. */
int mbir_selftest_bounded_wait(long long max_cycles);

const char* mbir_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* MBIR_H */
