// Internal definitions shared by the library's host setup and CUDA kernels.
//
// Device units: time in samples (1 / fs), lengths in metres.  A leg's ray
// parameter p is in samples per metre, so sin(theta_l) = p * k_l with
// k_l = c_l / fs, and the slowness of layer l is s_l = fs / c_l.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/mbir.h"

namespace mbir {

constexpr int kMaxLayers = MBIR_MAX_LAYERS;
constexpr int kBisect = 22;          // FP32 bisection steps on p (bracket / 2^22)

// Per-geometry constants, passed to kernels by value.
struct GeomParams {
    int L, W, H, n_tx, n_rx, K, M, Mp;
    int Tw, Tw4, Q, G, Gt;           // Gt = table gamma planes (max(G-1, 1))
    int mode, precision;
    int npos, nh;                     // distinct transducer positions, distinct |h| (TAB)
    int beta_int;                     // >= 0: beta is this integer; -1: use powf
    float beta;
    float gscale;                     // (G-1) / gamma_max (gamma bins per second)
    float inv_gscale;
    float k[kMaxLayers];              // c_l / fs  (m per sample)
    float2 kd[kMaxLayers];            // c_l / fs as double-float
    float2 s2[kMaxLayers];            // (fs / c_l)^2 as double-float
    float2 eta[kMaxLayers];           // full layer thickness as double-float
    float alpha_c[kMaxLayers];        // alpha_l (s/m) * gscale: gamma-bin units per metre
    int n_seg;                        // layer segments among image rows
    int seg_row[kMaxLayers + 1];      // first row of each segment, seg_row[n_seg] = H
    int apod_first;                   // eq. 12 with the first-layer angle instead of the angle sum
    float2 tilt_c, tilt_s;            // cos / sin of the transmitter firing angle (double-float)
};

// Per image row.
struct RowInfo {
    int nl;                           // layers crossed (eta > 0)
    float pmax;                       // fs / max crossed speed
    float2 eta_last;                  // eta of the deepest crossed layer (double-float)
    float tau;                        // interface transmittance product
    float tvert;                      // two-way vertical time (lower bound of T), samples
    float mrow;                       // unused by the operator (prior weight slot)
    int pad;
};

struct Leg {
    float Th, Tl;                     // travel time (double-float, samples)
    float g;                          // attenuation in gamma-bin units
    float phi;                        // cos^beta of the summed refraction angles
};

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum, FMA TwoProduct) and double-float
// arithmetic.  Intrinsics keep the compiler from contracting or reordering.
// ---------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ df df_mul(df a, df b)
{
    df p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b)
{
    df p = two_prod(a.hi, b);
    float e = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}

// sqrt of a non-negative double-float: IEEE sqrt of the head, one Newton step
__device__ __forceinline__ df df_sqrt(df a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    float r = __fsqrt_rn(a.hi);
    float e = __fadd_rn(__fmaf_rn(-r, r, a.hi), a.lo);
    return fast_two_sum(r, __fmul_rn(e, __fdividef(0.5f, r)));
}

__device__ __forceinline__ df df_div(df a, df b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_sub(a, df_mul_f(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

// c^beta in double-float for integer beta (binary powering), FP32 otherwise
__device__ __forceinline__ float pow_beta_df(df c, int beta_int, float beta)
{
    if (!(c.hi > 0.0f)) return 0.0f;
    if (beta_int >= 0) {
        df r = {1.0f, 0.0f}, b = c;
        int e = beta_int;
        while (e) {
            if (e & 1) r = df_mul(r, b);
            b = df_mul(b, b);
            e >>= 1;
        }
        return __fadd_rn(r.hi, r.lo);
    }
    return powf(c.hi, beta);
}

__device__ __forceinline__ float pow_beta(float c, int beta_int, float beta)
{
    if (!(c > 0.0f)) return 0.0f;
    if (beta_int >= 0) {
        float r = 1.0f, b = c;
        int e = beta_int;
        while (e) {
            if (e & 1) r *= b;
            b *= b;
            e >>= 1;
        }
        return r;
    }
    return powf(c, beta);
}

// |x_c - u| as double-float from double-float operands
__device__ __forceinline__ df abs_diff(float2 xc, float2 u)
{
    df s = two_sum(xc.x, -u.x);
    float e = __fadd_rn(s.lo, __fsub_rn(xc.y, u.y));
    df h = fast_two_sum(s.hi, e);
    if (h.hi < 0.0f) { h.hi = -h.hi; h.lo = -h.lo; }
    return h;
}

// ---------------------------------------------------------------------------
// One leg (Section 2, eq. 4-6) from a transducer at depth 0 to a voxel of row
// `ri` at lateral offset h >= 0.  The paper's binary search on theta_1 runs
// here on the ray parameter p = sin(theta_1) / c_1 (monotone in theta_1), in
// FP32 with a fixed step count so a warp stays in lockstep; one Newton step on
// X(p) = sum_l eta_l tan(theta_l) = h in double-float arithmetic then brings p
// to ~1e-13 relative.  The travel time uses the Legendre form
// T = p h + sum_l eta_l sqrt(s_l^2 - p^2) (stationary in p), the apodization
// cos^beta(sum theta_l) is built from the layer angles' cosines and sines by
// complex multiplication, all in double-float: beta = 8 multiplies the
// relative error of the cosine by eight.
// ---------------------------------------------------------------------------
template <int NL>
__device__ __forceinline__ Leg solve_leg(const GeomParams& P, const RowInfo& ri, df h, int tsign = 0)
{
    float eta[NL], kk[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        bool act = l < ri.nl;
        eta[l] = (l < ri.nl - 1) ? P.eta[l].x : (l == ri.nl - 1 ? ri.eta_last.x : 0.0f);
        kk[l] = act ? P.k[l] : 0.0f;
    }
    float lo = 0.0f, hi = ri.pmax;
#pragma unroll 2
    for (int it = 0; it < kBisect; ++it) {
        float mid = 0.5f * (lo + hi);
        float X = 0.0f;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            float t = mid * kk[l];
            float c2 = __fmaf_rn(-t, t, 1.0f);
            X = __fmaf_rn(eta[l] * t, rsqrtf(c2), X);
        }
        bool below = X < h.hi;
        lo = below ? mid : lo;
        hi = below ? hi : mid;
    }
    df p = {0.5f * (lo + hi), 0.0f};

    // Newton step in double-float: p -= (X(p) - h) / X'(p)
    if (h.hi > 0.0f) {
        df X = {0.0f, 0.0f};
        float dX = 0.0f;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            if (l < ri.nl) {
                float2 e2 = (l < ri.nl - 1) ? P.eta[l] : ri.eta_last;
                df e = {e2.x, e2.y};
                df t = df_mul(p, {P.kd[l].x, P.kd[l].y});
                df c = df_sqrt(df_sub({1.0f, 0.0f}, df_mul(t, t)));
                if (c.hi > 0.0f) {
                    X = df_add(X, df_mul(e, df_div(t, c)));
                    dX += e.hi * P.k[l] / (c.hi * c.hi * c.hi);
                }
            }
        }
        df diff = df_sub(X, h);
        if (dX > 0.0f && isfinite(diff.hi)) {
            float dp = __fdiv_rn(diff.hi, dX);
            if (fabsf(dp) < 1e-5f * p.hi + 1e-30f) p = df_add(p, {-dp, 0.0f});
        }
    }

    df T = df_mul(h, p);
    df p2 = df_mul(p, p);
    float g = 0.0f;
    df C = {1.0f, 0.0f}, Sn = {0.0f, 0.0f};
    df C1 = {1.0f, 0.0f}, S1 = {0.0f, 0.0f};                      // cos, sin of theta_1
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (l < ri.nl) {
            float2 e2 = (l < ri.nl - 1) ? P.eta[l] : ri.eta_last;
            df e = {e2.x, e2.y};
            df s2 = {P.s2[l].x, P.s2[l].y};
            df sq = df_sqrt(df_sub(s2, p2));
            T = df_add(T, df_mul(e, sq));
            df t = df_mul(p, {P.kd[l].x, P.kd[l].y});            // sin(theta_l)
            df c = df_sqrt(df_sub({1.0f, 0.0f}, df_mul(t, t)));   // cos(theta_l)
            g = __fmaf_rn(P.alpha_c[l] * eta[l], __frcp_rn(fmaxf(c.hi, 1e-30f)), g);  // alpha * path
            df Cn = df_sub(df_mul(C, c), df_mul(Sn, t));          // cos, sin of the angle sum
            Sn = df_add(df_mul(Sn, c), df_mul(C, t));
            C = Cn;
            if (l == 0) { C1 = c; S1 = t; }
        }
    }
    if (P.apod_first) { C = C1; Sn = S1; }
    if (tsign != 0) {
        // a transmitter tilted by psi toward +x: cos(s * angle - psi) = cos a cos psi + s sin a sin psi
        df a = df_mul(C, {P.tilt_c.x, P.tilt_c.y}), b = df_mul(Sn, {P.tilt_s.x, P.tilt_s.y});
        C = tsign > 0 ? df_add(a, b) : df_sub(a, b);
    }
    Leg out;
    out.Th = T.hi;
    out.Tl = T.lo;
    out.g = g;
    out.phi = pow_beta_df(C, P.beta_int, P.beta);
    return out;
}

// Tap parameters of one (pixel, A-scan) pair.  Taps are samples
// n = n0 + 1 + m, m = 0..Tw-1, at table coordinate q = m*Q + r with weight
// (1 - w1) on node q and w1 on node q + 1.  flag0 marks T exactly on a sample
// (the tap m = Tw-1 then sits at tau = t0 and is outside the open window).
struct Pair {
    int n0;
    int r, gi;
    float w0, w1;        // tau weights of nodes q and q + 1
    float psi;           // gamma weight of plane gi + 1
    float w;             // tau(l_v) * phi_tx * phi_rx
    bool flag0;
};

__device__ __forceinline__ Pair make_pair(const GeomParams& P, const Leg& tx, const Leg& rx, float tau)
{
    Pair o;
    df T = df_add({tx.Th, tx.Tl}, {rx.Th, rx.Tl});
    float n0f = floorf(T.hi);
    float f = __fadd_rn(__fsub_rn(T.hi, n0f), T.lo);
    if (f < 0.0f) { f += 1.0f; n0f -= 1.0f; }
    if (f >= 1.0f) { f -= 1.0f; n0f += 1.0f; }
    float a = f * (float)P.Q;
    if (a >= (float)P.Q) { n0f += 1.0f; f = 0.0f; a = 0.0f; }
    o.n0 = (int)n0f;
    float fl = floorf(a);
    int ia = (int)fl;
    float fa = a - fl;
    o.r = P.Q - 1 - ia;
    o.w1 = 1.0f - fa;
    o.w0 = fa;
    o.flag0 = (f == 0.0f);
    float gam = fminf(fmaxf(tx.g + rx.g, 0.0f), (float)(P.G - 1));
    int gi = (P.G > 1) ? min((int)gam, P.G - 2) : 0;
    o.gi = gi;
    o.psi = (P.G > 1) ? gam - (float)gi : 0.0f;
    o.w = tau * tx.phi * rx.phi;
    return o;
}

// Host-side launchers (apply.cu / map.cu)
struct GeomDev;
struct TsView;             // tensor-core apply views (tc_stream.cuh)
struct TbView;
}  // namespace mbir

// The geometry handle (opaque in the C ABI).
// Layout of the tensor-core A x (tc_stream.cuh): the table operand resident in shared memory, an FP32 sum
// tile of kwmax columns, the output row; the sums go to tensor memory as the MMA's A operand.
struct Tf4Layout {
    int parts;             // 2: FP32 form (two FP16 parts of the table and of the sums), 1: BF16 form
    int R;                 // phases per plane (Q + 1): column = plane * R + phase
    int kb;                // table operand columns: G * R rounded up to 16
    int ntap;              // MMA N: taps rounded up to 16
    int kwmax;             // widest column range of a tile that the sum tile holds (multiple of 16)
    int astride;           // FP32 row stride of the sums (floats, 4 mod 32)
    int texp;              // FP32 form: table operand = table x 2^texp (largest magnitude in [2^14, 2^15))
    int ylen;              // output samples held in shared memory (a ring)
    size_t bbytes;         // bytes of the table operand
    size_t off_part, off_rs, off_b, off_s, off_y, smem;
    bool ok;
};

// Layout of the tensor-core A^T (tc_stream.cuh): the table operand resident in shared memory, the
// residual windows of the current and the next item, the correlation tile of kwmax columns; the residual's
// Hankel tile goes to tensor memory as the MMA's A operand.
struct Tb4Layout {
    int parts;             // 2: FP32 form (two FP16 parts), 1: BF16 form
    int R, kb, ntap;       // as Tf4Layout
    int kwmax;             // widest column range of a tile that the correlation tile holds (multiple of 16)
    int cstride;           // FP32 row stride of the correlation tile (floats, 4 mod 32)
    int ewin;              // floats of one residual window (128 + taps, padded)
    int texp;              // FP32 form: table operand = table x 2^texp
    size_t bbytes;         // bytes of the table operand (table rows x taps, K-major)
    size_t off_e, off_b, off_c, smem;
    bool ok;
};

struct mbir_geometry {
    int device;
    mbir::GeomParams P;
    mbir::RowInfo* d_rows;
    float2* d_colx;        // W pixel-centre laterals (double-float)
    float2* d_pos;         // npos distinct transducer laterals (double-float)
    int* d_txpos;          // n_tx position index per Tx
    int* d_rxpos;          // K position index per A-scan receiver
    float2* d_tab;         // Gt x (Q+1) x Tw4 pulse table, float2 = (plane g, plane g+1)
    __nv_bfloat162* d_tab_bf16;
    float4* d_legs;        // TAB: H x nh legs
    int* d_hidx;           // TAB: npos x W index into the |h| list
    float* d_direct;       // n_rx x Mp direct-arrival columns (eq. 1)
    float* d_dinv;         // n_rx: 1 / |d_j|^2 (0 if empty)
    int* d_status;         // device error flag (bounded waits)
    // reconstruction workspace (grown on demand)
    float* w_e;            // K x Mp projected residual
    float* w_q;            // K x Mp P A d
    float* w_b;            // N
    float* w_grad;         // N
    float* w_gprev;        // N
    float* w_d;            // N
    double* w_part;        // reduction partials
    double* w_scal;        // scalar slots
    __nv_bfloat16* w_ebf;  // K x Mp BF16 copy of e (BF16 precision)
    size_t part_len;
    size_t bytes;
    double* tab_host;
    size_t tab_len;
    float* w_msq;          // H: sqrt(m_s) of eq. 17 for the current prior
    float* w_d2;           // N: second direction buffer (ping-pong)
    float* w_xalt;         // N: second image buffer of the fused update-and-prior stencil (ping-pong)
    float* w_y;            // K x M staging for host-buffer calls
    float* w_x;            // N staging for host-buffer calls
    float* w_g;            // K staging for host-buffer calls
    double* w_hist;        // 2 x hist_len: cost and gradient norm per iteration
    int hist_len;
    double gamma_max;
    double fs;
    double z0, pitch;
    // A^T r work list: (tile row, tile column, A-scan range, group) and per-group partial images
    int n_sm;
    int bwd_halves, bwd_stages;   // A^T r tile workers per CTA and residual ring depth
    int n_items, n_groups;
    int4* d_items;         // ordered by decreasing estimated cost
    float* w_bpart;
    int* d_bwd_counter;    // work counter of the A^T r launch
    float* h_bwd_cost;     // host copy: estimated A^T r cost per (16-row tile, 32-column tile, Tx position)
    int bwd_ntc;           // 32-column tiles per row of tiles
    // TAB-mode A x records sorted by first tap sample (see forward_tab.cu); with the tensor-core applies the
    // sorted records are replaced by their packed form (tc_apply.cuh), on the same per-A-scan offsets
    long long* d_rec_off;
    int2* d_rec_key;
    float4* d_rec_w;
    uint2* d_tc_key;       // packed records: keys
    void* d_tc_w;          // and weights (uint2 in the FP32 form, uint32 in the BF16 form)
    int2* d_runs;
    int fwd_sub;           // 32-sample spans per A x window (autotuned)
    double fwd_tune_ms[3]; // measured A x times of windows of 1, 2, 4 spans
    long long n_win;       // K x windows
    int* d_win_order;      // windows by decreasing record count
    int* h_win_cost;       // host copy: records per window (K x windows), for work partitioning
    float* h_tvert;        // host copy: vertical two-way time per image row (samples)
    int* d_win_counter;    // work counter of the A x launch
    // tensor-core A^T (see tc_adjoint.cu, tc_stream.cuh)
    int* d_tc_tile;        // first record of every 128-sample tile, K x (tiles + 1)
    unsigned long long* w_tc_acc;   // per pixel: fixed-point sum, N + 1 (the last word: bits of max |e|)
    float tc_bound;        // scale bound of the fixed-point sums (build_tc_adjoint)
    int* d_tc_counter;
    // tensor-core A x (see tc_stream.cuh, tc_fwd_stream.cu)
    mbir::TsView* d_tf_view;   // fwd_tcs_kernel's view without the per-call fields (device memory)
    mbir::TbView* d_tb_view;   // bwd_tcs_kernel's view without the residual (device memory)
    int* d_tf_order;       // A-scans by decreasing record count
    int* d_tf_counter;
    Tf4Layout tf4;
    uint4* d_tf4_bop;      // table operand (taps x columns plane * (Q + 1) + phase, K-major; FP32: two parts)
    uint32_t* d_tf4_crange;// per (A-scan, tile of 128 n0): first | end column << 16 of the planes its records reach
    int* d_tf4_split;      // per (A-scan, tile): the 17 boundaries of the warps' parts (record offsets)
    int tf4_wmax;          // widest column range of a tile
    // tensor-core A^T (see tc_stream.cuh); uses the tile offsets, slots and contributions of build_tc_adjoint
    Tb4Layout tb4;
    int tc_fvar, tc_bvar;  // variants of the tensor-core A x and A^T pools (tc_stream.cuh), chosen by timing
    double tc_tune_ms[4];  // their measured times: A x variant 0, 1, A^T variant 0, 1 (0 when not timed)
    uint4* d_tb4_bop;      // table operand (table rows plane * (Q + 1) + phase x taps, K-major; FP32: two parts)
    long long n_records;
    // |A_v|^2 per pixel for the coordinate descent (computed on its first call)
    float* w_colnorm;
    // coordinate descent work lists for colour spacing icd_s (built on the first call with that spacing):
    // A^T items per colour over lattice tiles, and (with records) per-colour record lists for A x
    int icd_s;
    int icd_groups;             // A-scan chunks of the colour A^T items
    int* h_icd_item_off;        // host: s^2 + 1 offsets into d_icd_items
    int4* d_icd_items;
    float* w_icd_bpart;         // icd_groups x N partial images
    size_t icd_bytes;
    long long* d_icd_rec_off;   // s^2 x (K + 1) absolute record offsets
    int2* d_icd_rec_key;
    float4* d_icd_rec_w;
    int2* d_icd_runs;           // s^2 x K x spans
    int* d_icd_win;             // non-empty windows of every colour, largest first
    long long* h_icd_win_off;   // host: s^2 + 1 offsets into d_icd_win
    int icd_win_sub;            // spans per window of those lists
    size_t icd_rec_bytes;
    void* icd_exec;             // captured sweep (cudaGraphExec_t) and what it was captured for
    double icd_exec_key[8];
    void* icd_stream;           // capture stream (cudaStream_t)
    // profiling of the apply kernels inside mbir_reconstruct
    int prof;
    void* prof_state;      // host-side event lists (see map.cu)
    long long prof_nf, prof_nb;
    double prof_fms, prof_bms;
};

namespace mbir {
// launchers implemented in apply.cu
cudaError_t launch_build_legs(const mbir_geometry* g, const int* d_hsign, const float2* d_hvals, cudaStream_t st);
cudaError_t launch_backproject(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf,
                               float* b, cudaStream_t st);
cudaError_t launch_forward(const mbir_geometry* g, const float* x, float* y_f32, __nv_bfloat16* y_bf16,
                           int out_stride, cudaStream_t st);
cudaError_t launch_pad_rows(const mbir_geometry* g, const void* src, int src_bf16, float* dst_pad,
                            cudaStream_t st);
cudaError_t launch_pair_quantities(const mbir_geometry* g, const int* pix, const int* k, int n,
                                   double* T, float* gam, float* w, cudaStream_t st);
void prof_release(mbir_geometry* g);
cudaError_t launch_project_rows(const mbir_geometry* g, const void* src, int src_bf16, int sin, const float* sub,
                                int ssub, float* dst, int sout, float* gk, double* part, cudaStream_t st);
cudaError_t launch_to_bf16(const float* src, __nv_bfloat16* dst, long long n, cudaStream_t st);
void compute_msq(const mbir_geometry* g, const mbir_prior* pr, float* out);
cudaError_t launch_count_taps(const mbir_geometry* g, unsigned long long* d_out, cudaStream_t st);
cudaError_t build_sorted_records(mbir_geometry* g, cudaStream_t st, size_t cap_bytes);
cudaError_t tune_forward_window(mbir_geometry* g, cudaStream_t st);
cudaError_t launch_forward_sorted(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                                  cudaStream_t st);
size_t backproject_smem(const mbir_geometry* g);
bool backproject_config(const GeomParams& P, int* halves, int* stages);
int backproject_tile_rows();
cudaError_t backproject_tile_costs(const mbir_geometry* g, int ntr, int ntc, float* h_cost, cudaStream_t st);
cudaError_t launch_backproject_partials(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf,
                                        float* b, float* partial, cudaStream_t st);
cudaError_t load_backproject_partials(const mbir_geometry* g);
cudaError_t load_pad_rows();
cudaError_t noalloc_prepare(const mbir_geometry* g);
size_t forward_smem(const mbir_geometry* g, int* cb_out);
cudaError_t build_tc_adjoint(mbir_geometry* g, cudaStream_t st);
void free_tc_adjoint(mbir_geometry* g);
Tf4Layout tf4_layout(const GeomParams& P, int kwmax);
cudaError_t build_tc_forward_stream(mbir_geometry* g, cudaStream_t st);
Tb4Layout tb4_layout(const GeomParams& P, int kwmax);
cudaError_t build_tc_adjoint_stream(mbir_geometry* g, cudaStream_t st);
cudaError_t tune_tc_applies(mbir_geometry* g, cudaStream_t st);
cudaError_t launch_backproject_tcs_update(const mbir_geometry* g, float* e, __nv_bfloat16* ebf, const float* q,
                                          const double* sc, int alpha_slot, float* b, cudaStream_t st);
cudaError_t launch_backproject_tcs(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf, float* b,
                                   cudaStream_t st);
cudaError_t launch_forward_tcs(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                               cudaStream_t st);
cudaError_t launch_column_norms(const mbir_geometry* g, float* out, cudaStream_t st);
cudaError_t build_colour_records(mbir_geometry* g, int s, cudaStream_t st);
cudaError_t launch_forward_colour(const mbir_geometry* g, int c, const float* x, float* yf, int stride,
                                  cudaStream_t st);
cudaError_t launch_backproject_lattice(const mbir_geometry* g, const int4* items, int nitems, int ngroups, int3 lat,
                                       float* partial, const float* e_pad, const __nv_bfloat16* e_bf, float* b,
                                       cudaStream_t st);
cudaError_t build_icd_lists(mbir_geometry* g, int s, cudaStream_t st);
void free_icd_lists(mbir_geometry* g);
}  // namespace mbir
