// Host side of the library: argument validation, the pulse table (built once
// in FP64 by FFT), per-row and per-transducer tables, device uploads, the
// leg table of TAB mode, and the C ABI entry points that manage handles.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "mbir_internal.h"

using mbir::GeomParams;
using mbir::RowInfo;

namespace {

constexpr double kPi = 3.14159265358979323846;

float2 split_df(double v)
{
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    return make_float2(hi, lo);
}

// iterative radix-2 complex FFT (sign -1 forward, +1 inverse, unnormalised)
void fft(std::vector<std::complex<double>>& a, int sign)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        double ang = sign * 2.0 * kPi / (double)len;
        for (size_t i = 0; i < n; i += len) {
            for (size_t k = 0; k < len / 2; ++k) {
                std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
                std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

struct Derived {
    int Tw, G, Q;
    double sigma, t0, tc, gmax;
};

int layer_of(const mbir_geometry_desc* d, double z, double* eta, int* nl_out)
{
    double top = 0.0;
    int lv = 0;
    for (int l = 0; l < d->n_layers; ++l) {
        if (l == d->n_layers - 1 || z < top + d->thickness_m[l]) { lv = l; break; }
        top += d->thickness_m[l];
    }
    for (int l = 0; l < lv; ++l) eta[l] = d->thickness_m[l];
    eta[lv] = z - top;
    *nl_out = eta[lv] > 0.0 ? lv + 1 : lv;
    return lv;
}

int validate(const mbir_geometry_desc* d)
{
    if (!d) return MBIR_ERR_INVALID_ARG;
    if (d->n_layers < 1 || d->n_layers > MBIR_MAX_LAYERS) return MBIR_ERR_INVALID_ARG;
    for (int l = 0; l < d->n_layers; ++l) {
        if (!(d->thickness_m[l] > 0) || !(d->speed_mps[l] > 0) || !(d->density_kgm3[l] > 0) ||
            !(d->atten_np_per_mhz_m[l] >= 0) || !std::isfinite(d->thickness_m[l]) ||
            !std::isfinite(d->speed_mps[l]) || !std::isfinite(d->atten_np_per_mhz_m[l]))
            return MBIR_ERR_INVALID_ARG;
    }
    if (d->img_w < 1 || d->img_h < 1 || d->img_h > 32767 || !(d->pitch_m > 0) || !(d->img_z0_m >= 0) ||
        !std::isfinite(d->img_x0_m))
        return MBIR_ERR_INVALID_ARG;
    if (d->n_tx < 1 || d->n_rx < 1 || d->n_tx > 65535 || !d->tx_x_m || !d->rx_offset_m) return MBIR_ERR_INVALID_ARG;
    if (!(d->fs_hz > 0) || d->n_samples < 1 || !(d->fc_hz > 0) || !(d->n_cycles > 0) || !(d->beta >= 0))
        return MBIR_ERR_INVALID_ARG;
    if (d->gamma_max_s < 0 || d->gamma_bins < 0 || d->gamma_bins == 1 || d->phases < 0 ||
        d->gamma_bins > 64 || d->phases > 64)
        return MBIR_ERR_INVALID_ARG;
    if (d->precision != MBIR_PREC_FP32 && d->precision != MBIR_PREC_BF16) return MBIR_ERR_INVALID_ARG;
    if (d->mode < MBIR_MODE_AUTO || d->mode > MBIR_MODE_TAB) return MBIR_ERR_INVALID_ARG;
    if (!std::isfinite(d->firing_angle_rad) || !(std::fabs(d->firing_angle_rad) < 0.5 * M_PI) ||
        (d->apodization != MBIR_APOD_ANGLE_SUM && d->apodization != MBIR_APOD_FIRST_ANGLE))
        return MBIR_ERR_INVALID_ARG;
    for (int i = 0; i < d->n_tx; ++i) if (!std::isfinite(d->tx_x_m[i])) return MBIR_ERR_INVALID_ARG;
    for (int j = 0; j < d->n_rx; ++j) if (!std::isfinite(d->rx_offset_m[j])) return MBIR_ERR_INVALID_ARG;
    long long N = (long long)d->img_w * d->img_h;
    long long K = (long long)d->n_tx * d->n_rx;
    if (N > (1LL << 30) || K * (long long)d->n_samples > (1LL << 31) || d->n_samples > 60000 || K > 65535)
        return MBIR_ERR_INVALID_ARG;
    return MBIR_OK;
}

Derived derive(const mbir_geometry_desc* d)
{
    Derived r;
    r.sigma = d->n_cycles / (2.0 * std::sqrt(2.0 * std::log(2.0)) * d->fc_hz);
    r.Tw = (int)std::ceil(8.0 * r.sigma * d->fs_hz);
    r.t0 = r.Tw / d->fs_hz;
    r.tc = 0.5 * r.t0;
    r.Q = d->phases > 0 ? d->phases : 16;
    int G = d->gamma_bins > 0 ? d->gamma_bins : 16;
    if (d->gamma_max_s > 0) {
        r.gmax = d->gamma_max_s;
    } else {
        double eta[MBIR_MAX_LAYERS];
        int nl;
        layer_of(d, d->img_z0_m + (d->img_h - 0.5) * d->pitch_m, eta, &nl);
        double s = 0;
        for (int l = 0; l < nl; ++l) s += d->atten_np_per_mhz_m[l] * 1e-6 * eta[l];
        r.gmax = 4.0 * s;
    }
    r.G = r.gmax > 0 ? G : 1;
    return r;
}

// h(gamma_g, q / (fs Q)) for g < G, q <= Q*Tw: the sampled pulse's spectrum,
// attenuated by exp(-gamma |f|) (eq. 9), transformed back.  The sample grid
// is the table's own tau grid, so no interpolation is involved.
std::vector<double> pulse_table(const mbir_geometry_desc* d, const Derived& D)
{
    const int nq = D.Q * D.Tw + 1;
    const double dt = 1.0 / (d->fs_hz * D.Q);
    size_t n = 1;
    while (n < (size_t)16 * nq) n <<= 1;
    std::vector<std::complex<double>> s(n);
    for (size_t k = 0; k < n; ++k) {
        double t = (k < n / 2) ? k * dt : ((double)k - (double)n) * dt;
        double u = t - D.tc;
        s[k] = std::exp(-u * u / (2.0 * D.sigma * D.sigma)) * std::cos(2.0 * kPi * d->fc_hz * u);
    }
    fft(s, -1);
    std::vector<double> tab((size_t)D.G * nq);
    std::vector<std::complex<double>> a(n);
    const double df_ = 1.0 / (n * dt);
    for (int g = 0; g < D.G; ++g) {
        double gam = D.G > 1 ? g * D.gmax / (D.G - 1) : 0.0;
        for (size_t k = 0; k < n; ++k) {
            double f = (k <= n / 2) ? k * df_ : ((double)k - (double)n) * df_;
            a[k] = s[k] * std::exp(-gam * std::fabs(f));
        }
        fft(a, +1);
        for (int q = 0; q < nq; ++q) tab[(size_t)g * nq + q] = a[q].real() / (double)n;
    }
    return tab;
}

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t count, size_t* bytes)
{
    size_t b = sizeof(T) * std::max<size_t>(count, 1);
    cudaError_t e = cudaMalloc((void**)dst, b);
    if (e != cudaSuccess) return e;
    *bytes += b;
    if (count) e = cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
    return e;
}

void free_geometry(mbir_geometry* g)
{
    if (!g) return;
    void* ptrs[] = {g->d_rows, g->d_colx, g->d_pos, g->d_txpos, g->d_rxpos, g->d_tab, g->d_tab_bf16,
                    g->d_legs, g->d_hidx, g->d_direct, g->d_dinv, g->d_status, g->w_e, g->w_q,
                    g->w_b, g->w_grad, g->w_gprev, g->w_d, g->w_part, g->w_scal, g->w_ebf,
                    g->w_msq, g->w_d2, g->w_xalt, g->w_y, g->w_x, g->w_g, g->w_hist, g->d_items, g->w_bpart,
                    g->d_rec_off, g->d_rec_key, g->d_rec_w, g->d_tc_key, g->d_tc_w, g->d_runs, g->d_win_order, g->d_win_counter,
                    g->d_bwd_counter, g->d_tc_tile, g->w_tc_acc,
                    g->d_tc_counter, g->d_tf_order, g->d_tf_counter, g->w_colnorm,
                    g->d_tf4_bop, g->d_tf4_crange, g->d_tf4_split, g->d_tb4_bop, g->d_tf_view, g->d_tb_view};
    for (void* p : ptrs) if (p) cudaFree(p);
    mbir::free_icd_lists(g);
    if (g->icd_stream) cudaStreamDestroy((cudaStream_t)g->icd_stream);
    mbir::prof_release(g);
    free(g->tab_host);
    free(g->h_win_cost);
    free(g->h_tvert);
    free(g->h_bwd_cost);
    delete g;
}

int cuda_err(cudaError_t e) { return e == cudaErrorMemoryAllocation ? MBIR_ERR_OOM : MBIR_ERR_CUDA; }

}  // namespace

extern "C" {

const char* mbir_error_string(int code)
{
    switch (code) {
    case MBIR_OK: return "ok";
    case MBIR_ERR_INVALID_ARG: return "invalid argument";
    case MBIR_ERR_OOM: return "out of memory";
    case MBIR_ERR_CUDA: return "CUDA error";
    case MBIR_ERR_NONFINITE: return "non-finite data or iterate";
    case MBIR_ERR_TIMEOUT: return "bounded wait timed out";
    case MBIR_ERR_BUSY: return "over the memory budget";
    case MBIR_ERR_UNSUPPORTED: return "unsupported option for this geometry";
    case MBIR_ERR_CANCELLED: return "cancelled";
    case MBIR_ERR_NOT_READY: return "not ready";
    default: return "unknown error";
    }
}

int mbir_create_geometry(const mbir_geometry_desc* d, void* stream, mbir_geometry** out)
{
    if (!out) return MBIR_ERR_INVALID_ARG;
    int rc = validate(d);
    if (rc != MBIR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Derived D = derive(d);
    mbir_geometry* g = new mbir_geometry();
    memset(g, 0, sizeof(*g));
    cudaGetDevice(&g->device);
    GeomParams& P = g->P;
    P.L = d->n_layers;
    P.W = d->img_w;
    P.H = d->img_h;
    P.n_tx = d->n_tx;
    P.n_rx = d->n_rx;
    P.K = d->n_tx * d->n_rx;
    P.M = d->n_samples;
    P.Tw = D.Tw;
    P.Tw4 = (D.Tw + 3) & ~3;
    P.Mp = (P.M + P.Tw4 + 8 + 7) & ~7;
    P.Q = D.Q;
    P.G = D.G;
    P.Gt = D.G > 1 ? D.G - 1 : 1;
    P.precision = d->precision;
    double bi = std::round(d->beta);
    P.beta_int = (std::fabs(d->beta - bi) == 0.0 && bi <= 64) ? (int)bi : -1;
    P.beta = (float)d->beta;
    P.apod_first = d->apodization == MBIR_APOD_FIRST_ANGLE ? 1 : 0;
    P.tilt_c = split_df(std::cos(d->firing_angle_rad));
    P.tilt_s = split_df(std::sin(d->firing_angle_rad));
    g->gamma_max = D.gmax;
    g->fs = d->fs_hz;
    g->z0 = d->img_z0_m;
    g->pitch = d->pitch_m;
    double gscale = (D.G > 1) ? (D.G - 1) / D.gmax : 0.0;
    P.gscale = (float)gscale;
    P.inv_gscale = (float)(gscale > 0 ? 1.0 / gscale : 0.0);
    for (int l = 0; l < mbir::kMaxLayers; ++l) {
        if (l < d->n_layers) {
            double c = d->speed_mps[l];
            P.k[l] = (float)(c / d->fs_hz);
            P.kd[l] = split_df(c / d->fs_hz);
            P.s2[l] = split_df((d->fs_hz / c) * (d->fs_hz / c));
            P.eta[l] = split_df(d->thickness_m[l]);
            P.alpha_c[l] = (float)(d->atten_np_per_mhz_m[l] * 1e-6 * gscale);
        } else {
            P.k[l] = 0.f;
            P.kd[l] = make_float2(0.f, 0.f);
            P.s2[l] = make_float2(0.f, 0.f);
            P.eta[l] = make_float2(0.f, 0.f);
            P.alpha_c[l] = 0.f;
        }
    }

    size_t bytes = 0;
    cudaError_t ce = cudaSuccess;
    std::vector<RowInfo> rows(P.H);
    int prev_lv = -1;
    P.n_seg = 0;
    for (int r = 0; r < P.H; ++r) {
        double z = d->img_z0_m + (r + 0.5) * d->pitch_m;
        double eta[MBIR_MAX_LAYERS];
        int nl;
        int lv = layer_of(d, z, eta, &nl);
        if (lv != prev_lv) {
            P.seg_row[P.n_seg++] = r;
            prev_lv = lv;
        }
        RowInfo& ri = rows[r];
        ri.nl = nl;
        double cmax = 0, tv = 0;
        for (int l = 0; l < nl; ++l) {
            cmax = std::max(cmax, d->speed_mps[l]);
            tv += 2.0 * eta[l] / d->speed_mps[l];
        }
        ri.pmax = (float)(cmax > 0 ? d->fs_hz / cmax : 0.0);
        ri.eta_last = split_df(nl > 0 ? eta[nl - 1] : 0.0);
        double tau = 1.0;
        for (int l = 1; l <= lv; ++l) {
            double z1 = d->density_kgm3[l - 1] * d->speed_mps[l - 1];
            double z2 = d->density_kgm3[l] * d->speed_mps[l];
            tau *= 4.0 * z1 * z2 / ((z1 + z2) * (z1 + z2));
        }
        ri.tau = (float)tau;
        ri.tvert = (float)(tv * d->fs_hz);
        ri.mrow = 0.f;
        ri.pad = 0;
    }
    P.seg_row[P.n_seg] = P.H;
    g->h_tvert = (float*)malloc(sizeof(float) * P.H);
    if (!g->h_tvert) { free_geometry(g); return MBIR_ERR_OOM; }
    for (int r = 0; r < P.H; ++r) g->h_tvert[r] = rows[r].tvert;

    // pixel-centre laterals and distinct transducer positions
    std::vector<float2> colx(P.W);
    for (int c = 0; c < P.W; ++c) colx[c] = split_df(d->img_x0_m + (c + 0.5) * d->pitch_m);
    std::vector<double> allpos;
    for (int i = 0; i < P.n_tx; ++i) {
        allpos.push_back(d->tx_x_m[i]);
        for (int j = 0; j < P.n_rx; ++j) allpos.push_back(d->tx_x_m[i] + d->rx_offset_m[j]);
    }
    std::vector<double> pos(allpos);
    std::sort(pos.begin(), pos.end());
    pos.erase(std::unique(pos.begin(), pos.end()), pos.end());
    P.npos = (int)pos.size();
    auto pos_index = [&](double u) {
        return (int)(std::lower_bound(pos.begin(), pos.end(), u) - pos.begin());
    };
    std::vector<int> txpos(P.n_tx), rxpos(P.K);
    for (int i = 0; i < P.n_tx; ++i) {
        txpos[i] = pos_index(d->tx_x_m[i]);
        for (int j = 0; j < P.n_rx; ++j) rxpos[i * P.n_rx + j] = pos_index(d->tx_x_m[i] + d->rx_offset_m[j]);
    }
    // a tilted transmitter's legs weigh differently from a receiver's at the same place:
    // its positions get entries of their own, whose legs depend on the sign of x_c - u
    const bool tilted = d->firing_angle_rad != 0.0;
    const int nshared = P.npos;
    if (tilted) {
        for (int i = 0; i < P.n_tx; ++i) {
            pos.push_back(d->tx_x_m[i]);
            txpos[i] = P.npos++;
        }
    }
    std::vector<float2> posdf(P.npos);
    for (int a = 0; a < P.npos; ++a) posdf[a] = split_df(pos[a]);

    // pulse table and its kernel layout
    std::vector<double> tab = pulse_table(d, D);
    const int nq = D.Q * D.Tw + 1;
    g->tab_len = tab.size();
    g->tab_host = (double*)malloc(sizeof(double) * tab.size());
    memcpy(g->tab_host, tab.data(), sizeof(double) * tab.size());
    const int R = D.Q + 1;
    const int S = P.Tw4 + 1;            // odd row stride: phases start on distinct bank pairs
    std::vector<float2> ktab((size_t)P.Gt * R * S);
    std::vector<__nv_bfloat162> ktab_bf(ktab.size());
    for (int gi = 0; gi < P.Gt; ++gi)
        for (int r = 0; r < R; ++r)
            for (int m = 0; m < S; ++m) {
                int q = m * D.Q + r;
                float a = 0.f, b = 0.f;
                if (m < D.Tw && q < nq) {
                    a = (float)tab[(size_t)gi * nq + q];
                    b = (float)tab[(size_t)(D.G > 1 ? gi + 1 : gi) * nq + q];
                }
                size_t idx = ((size_t)gi * R + r) * S + m;
                ktab[idx] = make_float2(a, b);
                ktab_bf[idx] = __floats2bfloat162_rn(a, b);
            }

    // direct-arrival columns (eq. 1): unattenuated pulse delayed by |o_j| / c_1
    std::vector<float> direct((size_t)P.n_rx * P.Mp, 0.f);
    std::vector<float> dinv(P.n_rx, 0.f);
    if (d->direct_arrival) {
        for (int j = 0; j < P.n_rx; ++j) {
            double T = std::fabs(d->rx_offset_m[j]) / d->speed_mps[0];
            double ss = 0;
            for (int n = 0; n < P.M; ++n) {
                double tau = n / d->fs_hz - T;
                double v = 0;
                if (tau > 0 && tau < D.t0) {
                    double u = tau * d->fs_hz * D.Q;
                    int q = (int)std::floor(u);
                    if (q > nq - 2) q = nq - 2;
                    double ph = u - q;
                    v = (1 - ph) * tab[q] + ph * tab[q + 1];
                }
                direct[(size_t)j * P.Mp + n] = (float)v;
                ss += (double)(float)v * (double)(float)v;
            }
            dinv[j] = ss > 0 ? (float)(1.0 / ss) : 0.f;
        }
    }

    // TAB: distinct |x_c - u| values per (position, column)
    // legs are keyed by |x_c - u| for receivers and untilted transmitters, and by the
    // signed x_c - u for tilted transmitters (listed after the others); hsign: 0, +1, -1
    std::vector<int> hidx;
    std::vector<float2> hvals;
    std::vector<int> hsign;
    int mode = d->mode;
    if (tilted && mode == MBIR_MODE_OTF) { free_geometry(g); return MBIR_ERR_UNSUPPORTED; }
    {
        std::vector<double> hv;
        hv.reserve((size_t)P.npos * P.W);
        for (int a = 0; a < P.npos; ++a)
            for (int c = 0; c < P.W; ++c) {
                const double x = d->img_x0_m + (c + 0.5) * d->pitch_m - pos[a];
                hv.push_back(a < nshared ? std::fabs(x) : x);
            }
        const double tol = 1e-9 * d->pitch_m;
        auto uniq_of = [tol](std::vector<double> v) {
            std::sort(v.begin(), v.end());
            std::vector<double> u;
            for (double x : v)
                if (u.empty() || x - u.back() > tol) u.push_back(x);
            return u;
        };
        std::vector<double> u0 = uniq_of(std::vector<double>(hv.begin(), hv.begin() + (size_t)nshared * P.W));
        std::vector<double> u1 = uniq_of(std::vector<double>(hv.begin() + (size_t)nshared * P.W, hv.end()));
        size_t tab_bytes = (size_t)P.H * (u0.size() + u1.size()) * sizeof(float4);
        if (mode == MBIR_MODE_AUTO) mode = (tab_bytes <= ((size_t)4 << 30)) ? MBIR_MODE_TAB : MBIR_MODE_OTF;
        if (tilted && mode != MBIR_MODE_TAB) { free_geometry(g); return MBIR_ERR_UNSUPPORTED; }
        if (mode == MBIR_MODE_TAB) {
            auto nearest = [tol](const std::vector<double>& u, double x) {
                size_t i = std::lower_bound(u.begin(), u.end(), x - tol) - u.begin();
                if (i + 1 < u.size() && std::fabs(u[i + 1] - x) < std::fabs(u[i] - x)) ++i;
                return i;
            };
            hidx.resize(hv.size());
            for (size_t t = 0; t < hv.size(); ++t)
                hidx[t] = t < (size_t)nshared * P.W ? (int)nearest(u0, hv[t]) : (int)(u0.size() + nearest(u1, hv[t]));
            for (double x : u0) {
                hvals.push_back(split_df(x));
                hsign.push_back(0);
            }
            for (double x : u1) {
                hvals.push_back(split_df(std::fabs(x)));
                hsign.push_back(x >= 0.0 ? 1 : -1);
            }
            P.nh = (int)hvals.size();
        }
    }
    P.mode = mode;

#define UP(ptr, vec)                                                  \
    do {                                                              \
        ce = upload(&ptr, (vec).data(), (vec).size(), &bytes);        \
        if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); } \
    } while (0)
    UP(g->d_rows, rows);
    UP(g->d_colx, colx);
    UP(g->d_pos, posdf);
    UP(g->d_txpos, txpos);
    UP(g->d_rxpos, rxpos);
    ktab.resize((ktab.size() + 15) & ~(size_t)15, make_float2(0.f, 0.f));
    ktab_bf.resize((ktab_bf.size() + 31) & ~(size_t)31, __floats2bfloat162_rn(0.f, 0.f));
    UP(g->d_tab, ktab);
    UP(g->d_tab_bf16, ktab_bf);
    UP(g->d_direct, direct);
    UP(g->d_dinv, dinv);
    std::vector<int> status(4, 0);
    UP(g->d_status, status);
    if (mode == MBIR_MODE_TAB) {
        UP(g->d_hidx, hidx);
        float2* d_hv = nullptr;
        int* d_hs = nullptr;
        size_t tmpb = 0;
        ce = upload(&d_hv, hvals.data(), hvals.size(), &tmpb);
        if (ce == cudaSuccess) ce = upload(&d_hs, hsign.data(), hsign.size(), &tmpb);
        if (ce != cudaSuccess) { cudaFree(d_hv); free_geometry(g); return cuda_err(ce); }
        ce = cudaMalloc((void**)&g->d_legs, sizeof(float4) * (size_t)P.H * P.nh);
        if (ce != cudaSuccess) { cudaFree(d_hv); cudaFree(d_hs); free_geometry(g); return cuda_err(ce); }
        bytes += sizeof(float4) * (size_t)P.H * P.nh;
        ce = mbir::launch_build_legs(g, d_hs, d_hv, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        cudaFree(d_hv);
        cudaFree(d_hs);
        if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
    }
    if (!mbir::backproject_config(P, &g->bwd_halves, &g->bwd_stages)) {
        // the pulse table plus two residual rows do not fit in shared memory
        free_geometry(g);
        return MBIR_ERR_UNSUPPORTED;
    }
    {
        // A^T r work list: active 16-row tiles x 32-column tiles x transmitter groups,
        // about eight items per tile worker, ordered by decreasing estimated cost so
        // that the persistent workers, taking items from a shared counter, finish together
        cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, g->device);
        if (g->n_sm < 1) g->n_sm = 1;
        const int TR = mbir::backproject_tile_rows();
        const int ntr = (P.H + TR - 1) / TR, ntc = (P.W + 31) / 32;
        g->bwd_ntc = ntc;
        int active_tiles = 0;
        for (int tr = 0; tr < ntr; ++tr)
            if (rows[tr * TR].tvert < (float)(P.M - 1)) active_tiles += ntc;
        int ngroups = 1;
        if (active_tiles > 0) {
            ngroups = (8 * g->bwd_halves * g->n_sm + active_tiles - 1) / active_tiles;
            ngroups = std::max(1, std::min(ngroups, P.n_tx));
        }
        const int txg = (P.n_tx + ngroups - 1) / ngroups;
        ngroups = (P.n_tx + txg - 1) / txg;
        g->h_bwd_cost = (float*)malloc(sizeof(float) * (size_t)ntr * ntc * P.n_tx);
        if (!g->h_bwd_cost) { free_geometry(g); return MBIR_ERR_OOM; }
        ce = mbir::backproject_tile_costs(g, ntr, ntc, g->h_bwd_cost, st);
        if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
        std::vector<int4> items;
        std::vector<double> cost;
        for (int tr = 0; tr < ntr; ++tr) {
            if (!(rows[tr * TR].tvert < (float)(P.M - 1))) continue;
            for (int tc = 0; tc < ntc; ++tc)
                for (int gi = 0; gi < ngroups; ++gi) {
                    int t0 = gi * txg, t1 = std::min(P.n_tx, t0 + txg);
                    double c = 0;
                    for (int t = t0; t < t1; ++t) c += g->h_bwd_cost[((size_t)tr * ntc + tc) * P.n_tx + t];
                    items.push_back(make_int4(tr, tc, (t0 * P.n_rx) | ((t1 * P.n_rx) << 16), gi));
                    cost.push_back(c);
                }
        }
        std::vector<int> order(items.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        std::vector<int4> sorted(items.size());
        for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
        g->n_items = (int)sorted.size();
        g->n_groups = ngroups;
        UP(g->d_items, sorted);
        ce = cudaMalloc((void**)&g->d_bwd_counter, sizeof(int));
        if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
        ce = cudaMalloc((void**)&g->w_bpart, sizeof(float) * (size_t)ngroups * P.W * P.H);
        if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
        bytes += sizeof(float) * (size_t)ngroups * P.W * P.H + sizeof(int);
    }
#undef UP
    if (P.mode == MBIR_MODE_TAB && !(d->flags & MBIR_FLAG_NO_RECORDS)) {
        size_t freeb = 0, totalb = 0;
        cudaMemGetInfo(&freeb, &totalb);
        size_t cap = std::min<size_t>(freeb / 2, (size_t)64 << 30);
        ce = mbir::build_sorted_records(g, st, cap);
        if (ce == cudaErrorNotSupported) ce = cudaSuccess;     // keep the on-the-fly record path
        if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
        if (g->d_rec_key && !(d->flags & MBIR_FLAG_NO_TENSOR_CORES)) {
            // A x first: it leaves the records in its kernel's order, on which the adjoint's slots are built
            ce = mbir::build_tc_forward_stream(g, st);
            if (ce == cudaErrorNotSupported) ce = cudaSuccess;  // keep the CUDA-core A x
            if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
            ce = mbir::build_tc_adjoint(g, st);
            if (ce == cudaErrorNotSupported) ce = cudaSuccess;  // keep the CUDA-core adjoint
            if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
            ce = mbir::build_tc_adjoint_stream(g, st);
            if (ce == cudaErrorNotSupported) {                  // keep the CUDA-core A^T
                mbir::free_tc_adjoint(g);
                ce = cudaSuccess;
            }
            if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
        }
        // the tensor-core pools' variants are chosen by timing them once
        if (g->d_tf4_bop || g->d_tb4_bop) {
            ce = mbir::tune_tc_applies(g, st);
            if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
        }
        // the CUDA-core A x's window is tuned only when that kernel is the geometry's A x
        if (g->d_rec_key && !g->d_tf4_bop) {
            ce = mbir::tune_forward_window(g, st);
            if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
        }
    }
    // set-up of the allocation-free adjoint for this device (a no-op for geometries it does not take)
    ce = mbir::noalloc_prepare(g);
    if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
    ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { free_geometry(g); return cuda_err(ce); }
    g->bytes += bytes;          // the record and tensor-core tables added theirs already
    *out = g;
    return MBIR_OK;
}

int mbir_destroy_geometry(mbir_geometry* g)
{
    if (!g) return MBIR_OK;
    int cur;
    cudaGetDevice(&cur);
    if (cur != g->device) cudaSetDevice(g->device);
    free_geometry(g);
    if (cur != g->device) cudaSetDevice(cur);
    return MBIR_OK;
}

size_t mbir_geometry_bytes(const mbir_geometry* g) { return g ? g->bytes : 0; }

int mbir_set_tensor_core_variants(mbir_geometry* g, int forward_variant, int adjoint_variant)
{
    if (!g || forward_variant < -1 || forward_variant > 1 || adjoint_variant < -1 || adjoint_variant > 1)
        return MBIR_ERR_INVALID_ARG;
    if ((forward_variant >= 0 && !g->d_tf4_bop) || (adjoint_variant >= 0 && !g->d_tb4_bop)) return MBIR_ERR_UNSUPPORTED;
    if (forward_variant >= 0) g->tc_fvar = forward_variant;
    if (adjoint_variant >= 0) g->tc_bvar = adjoint_variant;
    return MBIR_OK;
}

int mbir_geometry_get_info(const mbir_geometry* g, mbir_geometry_info* info)
{
    if (!g || !info) return MBIR_ERR_INVALID_ARG;
    info->n_pixels = (int64_t)g->P.W * g->P.H;
    info->n_ascans = g->P.K;
    info->n_samples = g->P.M;
    info->pulse_support = g->P.Tw;
    info->gamma_bins = g->P.G;
    info->phases = g->P.Q;
    info->gamma_max_s = g->gamma_max;
    info->mode = g->P.mode;
    info->precision = g->P.precision;
    info->device_bytes = (int64_t)g->bytes;
    info->forward_window_spans = g->d_rec_key ? g->fwd_sub : 0;
    for (int c = 0; c < 3; ++c) info->forward_window_ms[c] = g->fwd_tune_ms[c];
    info->adjoint_groups = g->n_groups;
    info->adjoint_tensor_cores = g->d_tb4_bop ? 1 : 0;
    info->forward_tensor_cores = g->d_tf4_bop ? 1 : 0;
    const bool has_rec = g->d_rec_key || g->d_tc_key;
    info->n_records = has_rec ? g->n_records : 0;
    const size_t per = g->d_tc_key ? sizeof(uint2) + (g->P.precision == MBIR_PREC_BF16 ? 4 : 8)
                                   : sizeof(int2) + sizeof(float4);
    info->record_bytes = has_rec ? (int64_t)(per * (size_t)g->n_records) : 0;
    info->tc_forward_variant = g->tc_fvar;
    info->tc_adjoint_variant = g->tc_bvar;
    for (int c = 0; c < 4; ++c) info->tc_variant_ms[c] = g->tc_tune_ms[c];
    return MBIR_OK;
}

int mbir_pulse_table(const mbir_geometry* g, double* out_host, size_t n)
{
    if (!g || !out_host || n < g->tab_len) return MBIR_ERR_INVALID_ARG;
    memcpy(out_host, g->tab_host, sizeof(double) * g->tab_len);
    return MBIR_OK;
}

int mbir_pair_quantities(const mbir_geometry* g, const int32_t* pix_host, const int32_t* k_host,
                         int n, double* T_host, float* gamma_host, float* w_host)
{
    if (!g || n < 0 || (n > 0 && (!pix_host || !k_host || !T_host || !gamma_host || !w_host)))
        return MBIR_ERR_INVALID_ARG;
    if (n == 0) return MBIR_OK;
    long long N = (long long)g->P.W * g->P.H;
    for (int t = 0; t < n; ++t)
        if (pix_host[t] < 0 || pix_host[t] >= N || k_host[t] < 0 || k_host[t] >= g->P.K)
            return MBIR_ERR_INVALID_ARG;
    int *dp = nullptr, *dk = nullptr;
    double* dT = nullptr;
    float *dg = nullptr, *dw = nullptr;
    cudaError_t e = cudaMalloc(&dp, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dT, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dg, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dw, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dp, pix_host, sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, k_host, sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mbir::launch_pair_quantities(g, dp, dk, n, dT, dg, dw, 0);
    if (e == cudaSuccess) e = cudaMemcpy(T_host, dT, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(gamma_host, dg, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(w_host, dw, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaFree(dp);
    cudaFree(dk);
    cudaFree(dT);
    cudaFree(dg);
    cudaFree(dw);
    return e == cudaSuccess ? MBIR_OK : cuda_err(e);
}

}  // extern "C"
