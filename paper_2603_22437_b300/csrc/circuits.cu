// Plans (public circuit configuration + encoded constants) and the two
// circuits: the small FIR+DFT instance and the vital-sign chain.
//
// Vital chain (paper Sec. "Example Pipelines", Encrypted Vital Signs, with the
// depth accounting of Table 1), L0 = top level:
//   side branch  K1: p = Re^2 + Im^2 (L0-1), E = rotate-sum over frames;
//                K2: w = E^2 (L0-2); num = sum idx (.) w, den = sum 1 (.) w
//                (L0-3), rotate-sum over the bins of a frame.
//   main chain   K4: p (L0-1), m = p^2 (L0-2), I = sum_c m Re, Q = sum_c m Im
//                (L0-3), rotate-sum over bins; K5: FIR per band, BSGS with
//                hoisted baby steps shared by both bands (L0-4); K7:
//                y = Qf If' - If Qf', x = If If' + Qf Qf' (L0-5), third order
//                u = 3x^2 - y^2 (L0-6), 3 dphi = y u (L0-7); K3 narrowband
//                DFT of both bands in one BSGS product, Re rows at k and Im
//                rows at k + F_pad/2 (+1); |X|^2 (+2), halves and bands
//                merged by one rotate-and-add; square (+3); frequency
//                weights and band indicator (+4), rotate-sum.
// Slot layout: slot(t, r) = t R_c + r, F_pad = 2^ceil(log2 F), R_c = N/2 / F_pad.
//
// Gesture chain (Sec. "Example Pipelines", Encrypted Dynamic Radar
// Classification; Table 1 pipeline 2), L0 = top level: per ciphertext pair
// K3 Doppler DFT (block-diagonal BSGS, hoisted baby steps of Re and Im,
// L0-1), K1 p = Re^2 + Im^2 (L0-2), K6 notch mask (L0-3), w = p^4 (L0-5),
// feature p w (L0-6); frames summed (pairs added, then a rotate-and-sum
// over the frames sharing a ciphertext); FC1 with extended diagonals over
// every feature slot and a rotate-and-sum to one period (L0-7), + bias and
// the constant 1, square (L0-8); FC2 + square (L0-10); FC3 (L0-11).  Every
// pair of every window of the batch is one ciphertext of each launch.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <set>
#include <tuple>

#include "circuits.h"
#include "engine.h"
#include "hostmath.h"

namespace mmfhe {

static int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

static int ilog2(int x) {
    int r = 0;
    while ((1 << r) < x) r++;
    return r;
}

static std::pair<int, int> bsgs_split(int ndiag) {
    int D = next_pow2(ndiag);
    int lg = ilog2(D);
    int n1 = 1 << ((lg + 1) / 2);
    return {n1, D / n1};
}

std::vector<int> band_bins(int frames, int fs_mhz, int lo_mhz, int hi_mhz) {
    std::vector<int> out;
    for (int k = 0; k <= frames / 2; k++) {
        long long kf = (long long)k * fs_mhz;
        if ((long long)lo_mhz * frames <= kf && kf <= (long long)hi_mhz * frames) out.push_back(k);
    }
    return out;
}

// ---------------------------------------------------------------------------
// FP64 public constants (the library's own design)
// ---------------------------------------------------------------------------
static double sinc(double x) {
    if (x == 0.0) return 1.0;
    double px = M_PI * x;
    return std::sin(px) / px;
}

// Hamming-windowed-sinc bandpass, unit gain at the band centre.
std::vector<double> fir_bandpass(int taps, double f_lo, double f_hi, double fs) {
    std::vector<double> h(taps);
    double M = (taps - 1) / 2.0, a = f_lo / fs, b = f_hi / fs, fc = 0.5 * (a + b), g = 0.0;
    for (int k = 0; k < taps; k++) {
        double m = k - M;
        double w = 0.54 - 0.46 * std::cos(2 * M_PI * k / (taps - 1));
        h[k] = (2 * b * sinc(2 * b * m) - 2 * a * sinc(2 * a * m)) * w;
        g += h[k] * std::cos(2 * M_PI * fc * m);
    }
    for (double &x : h) x /= g;
    return h;
}

static double hann(int n, int N) { return 0.5 - 0.5 * std::cos(2 * M_PI * n / (N - 1)); }

// ---------------------------------------------------------------------------
// encoder: m = round_half_away(scale * tau^-1(z)), slot j <-> zeta^(5^j)
// ---------------------------------------------------------------------------
static void fft_inplace(std::vector<std::complex<double>> &a) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        double ang = -2 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len) {
            for (size_t j = 0; j < len / 2; j++) {
                std::complex<double> w(std::cos(ang * j), std::sin(ang * j));
                std::complex<double> u = a[i + j], v = a[i + j + len / 2] * w;
                a[i + j] = u + v;
                a[i + j + len / 2] = u - v;
            }
        }
    }
}

void encode_slots(const mmfhe_params &p, const double *slots, double scale, int level, uint64_t *out,
                  const double *imag) {
    const uint32_t N = 1u << p.log_n, n = N / 2;
    std::vector<std::complex<double>> Z(N);
    uint64_t e = 1;
    for (uint32_t j = 0; j < n; j++) {
        const std::complex<double> z(slots[j], imag ? imag[j] : 0.0);
        Z[(e - 1) / 2] = z;
        Z[(2 * N - e - 1) / 2] = std::conj(z);   // the conjugate-symmetric extension
        e = (e * 5) % (2 * N);
    }
    fft_inplace(Z);
    for (uint32_t k = 0; k < N; k++) {
        std::complex<double> tw(std::cos(-M_PI * k / N), std::sin(-M_PI * k / N));
        double m = (tw * Z[k]).real() / N * scale;
        double r = m >= 0 ? std::floor(m + 0.5) : -std::floor(-m + 0.5);
        if (std::fabs(r) >= 9.2e18) throw Error(MMFHE_ERR_BAD_ARG, "encode: value too large for the scale");
        int64_t c = (int64_t)r;
        for (int i = 0; i <= level; i++) {
            uint64_t q = p.q[i];
            uint64_t a = c >= 0 ? (uint64_t)c % q : (q - ((uint64_t)(-(c + 1)) + 1) % q) % q;
            out[(size_t)i * N + k] = a;
        }
    }
}

// ---------------------------------------------------------------------------
// plan structure
// ---------------------------------------------------------------------------
static void check_fc_cfg(const Context &c, const mmfhe_circuit_config &cfg) {
    const uint32_t D = cfg.bins, L = cfg.taps;
    if (D < 2 || (D & (D - 1)) || D > c.n / 2) throw Error(MMFHE_ERR_BAD_ARG, "FC width must be a power of two within the slots");
    if (L < 1 || L > 8) throw Error(MMFHE_ERR_BAD_ARG, "FC networks have 1..8 layers");
    for (uint32_t l = 0; l <= L; l++)
        if (cfg.fc_dims[l] < 1 || cfg.fc_dims[l] >= D) throw Error(MMFHE_ERR_BAD_ARG, "FC layer widths must be 1..D-1");
    if (c.L - 2 * (int)L + 1 < 0) throw Error(MMFHE_ERR_BAD_ARG, "not enough levels in the parameter set for this circuit");
}

static bool is_vital(const mmfhe_circuit_config &cfg) {
    return cfg.kind == MMFHE_CIRCUIT_VITAL || cfg.kind == MMFHE_CIRCUIT_VITAL_PER_FRAME;
}

// Levels the gesture chain's feature map takes: the paper's p (p^2)^2 three,
// the learned a p + b p^2 one.
static int gesture_feature_depth(const mmfhe_circuit_config &cfg) {
    return cfg.feature_map == MMFHE_FEATURE_LEARNED ? 1 : 3;
}

static void check_gesture_cfg(const Context &c, const mmfhe_circuit_config &cfg) {
    const uint64_t A = cfg.antennas, R = cfg.bins, D = cfg.chirps, W = cfg.fc_width;
    if (A < 1 || R < 1 || D < 2 || cfg.frames < 1) throw Error(MMFHE_ERR_BAD_ARG, "bad gesture sizes");
    const uint64_t ard = A * R * D;
    if ((uint64_t)next_pow2((int)std::min<uint64_t>(ard, 1u << 30)) > c.n / 2)
        throw Error(MMFHE_ERR_BAD_ARG, "a frame needs more slots than a ciphertext has");
    if (W < 2 || (W & (W - 1)) || W > (uint64_t)next_pow2((int)ard)) throw Error(MMFHE_ERR_BAD_ARG, "bad FC width");
    if (cfg.fc_dims[0] != ard) throw Error(MMFHE_ERR_BAD_ARG, "fc_dims[0] must be A R D");
    for (int l = 1; l <= 3; l++)
        if (cfg.fc_dims[l] < 1 || cfg.fc_dims[l] >= W) throw Error(MMFHE_ERR_BAD_ARG, "FC widths must be 1..fc_width-1");
    if (!(cfg.input_scale > 1.0)) throw Error(MMFHE_ERR_BAD_ARG, "input_scale must be the encryption scale");
    if (cfg.feature_map != MMFHE_FEATURE_POWER && cfg.feature_map != MMFHE_FEATURE_LEARNED)
        throw Error(MMFHE_ERR_BAD_ARG, "unknown feature map");
    if (c.L < 8 + gesture_feature_depth(cfg)) throw Error(MMFHE_ERR_BAD_ARG, "not enough levels for the gesture chain");
}

static void check_cfg(const Context &c, const mmfhe_circuit_config &cfg) {
    if (cfg.kind == MMFHE_CIRCUIT_FC) return check_fc_cfg(c, cfg);
    if (cfg.kind == MMFHE_CIRCUIT_GESTURE) return check_gesture_cfg(c, cfg);
    if (cfg.kind == MMFHE_CIRCUIT_VITAL_PER_FRAME) {
        if (cfg.frames < 2 || cfg.bins < 1 || cfg.taps < 1 || cfg.fs_mhz < 1 || cfg.taps > cfg.frames)
            throw Error(MMFHE_ERR_BAD_ARG, "bad circuit sizes");
        if ((uint32_t)next_pow2((int)cfg.bins) > c.n / 2) throw Error(MMFHE_ERR_BAD_ARG, "more bins than slots");
        if (cfg.taylor_order != 3 || cfg.num_bands != 2) throw Error(MMFHE_ERR_BAD_ARG, "per-frame chain: third order, two bands");
        if (c.L < 11) throw Error(MMFHE_ERR_BAD_ARG, "not enough levels for the vital chain");
        return;
    }
    if (cfg.kind != MMFHE_CIRCUIT_FIR_DFT && cfg.kind != MMFHE_CIRCUIT_VITAL) throw Error(MMFHE_ERR_BAD_ARG, "unknown circuit kind");
    if (cfg.frames < 2 || cfg.bins < 1 || cfg.taps < 1 || cfg.fs_mhz < 1) throw Error(MMFHE_ERR_BAD_ARG, "bad circuit sizes");
    int fpad = next_pow2((int)cfg.frames);
    if ((uint32_t)fpad > c.n / 2) throw Error(MMFHE_ERR_BAD_ARG, "window longer than the slot count");
    if (cfg.taps > cfg.frames) throw Error(MMFHE_ERR_BAD_ARG, "more taps than frames");
    if (cfg.kind == MMFHE_CIRCUIT_VITAL && !(cfg.taylor_order == 1 || cfg.taylor_order == 3))
        throw Error(MMFHE_ERR_BAD_ARG, "taylor_order must be 1 or 3");
    uint32_t nb = cfg.kind == MMFHE_CIRCUIT_VITAL ? 2 : 1;
    if (cfg.num_bands != nb) throw Error(MMFHE_ERR_BAD_ARG, "wrong number of bands");
}

uint64_t key_of(const mmfhe_const_key &k) {
    return ((uint64_t)k.tag << 48) | ((uint64_t)k.band << 40) | (uint64_t)k.index;
}

// Structurally present diagonals of a D x D layer d_in -> d_out: rows d_out
// and the constant row, columns d_in and the constant column.
static std::vector<int> present_diags(int D, int din, int dout) {
    std::vector<int> rows, cols;
    for (int i = 0; i < dout; i++) rows.push_back(i);
    for (int j = 0; j < din; j++) cols.push_back(j);
    rows.push_back(D - 1);
    cols.push_back(D - 1);
    std::set<int> ks;
    for (int i : rows)
        for (int j : cols) ks.insert(((j - i) % D + D) % D);
    return std::vector<int>(ks.begin(), ks.end());
}

// Structurally present diagonals of FC layer l.  Gesture plans: layers 1 and
// 2 on the period fc_width (layer 0 has every extended diagonal).
std::vector<int> fc_present(const mmfhe_circuit_config &cfg, int l) {
    if (cfg.kind == MMFHE_CIRCUIT_GESTURE)
        return present_diags((int)cfg.fc_width, (int)cfg.fc_dims[l], (int)cfg.fc_dims[l + 1]);
    return present_diags((int)cfg.bins, (int)cfg.fc_dims[l], (int)cfg.fc_dims[l + 1]);
}

static int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

static Plan *create_gesture_plan(Context &c, const mmfhe_circuit_config &cfg) {
    std::unique_ptr<Plan> p(new Plan());
    p->ctx = &c;
    p->cfg = cfg;
    const int L = c.L, D = (int)cfg.chirps, W = (int)cfg.fc_width, slots = (int)c.n / 2;
    const int ard = (int)(cfg.antennas * cfg.bins * cfg.chirps);
    p->ard_pad = next_pow2(ard);
    p->fpc = slots / p->ard_pad;
    p->pairs = ((int)cfg.frames + p->fpc - 1) / p->fpc;
    p->n1_k3 = bsgs_split(2 * D).first;
    p->n1_fc = bsgs_split(W).first;
    std::set<int32_t> rots;
    for (int delta = -(D - 1); delta < D; delta++) {
        if (cfg.complex_slots)
            p->keys.push_back(mmfhe_const_key{MMFHE_CONST_GDFT_W, 0, (uint32_t)(delta + D), (uint32_t)L});
        else
            for (uint32_t tag : {MMFHE_CONST_GDFT_C, MMFHE_CONST_GDFT_S, MMFHE_CONST_GDFT_MS})
                p->keys.push_back(mmfhe_const_key{tag, 0, (uint32_t)(delta + D), (uint32_t)L});
        rots.insert(norm_rot(c, floor_div(delta, p->n1_k3) * p->n1_k3));
    }
    if (cfg.complex_slots) rots.insert(MMFHE_ROT_CONJ);
    p->keys.push_back(mmfhe_const_key{MMFHE_CONST_NOTCH, 0, 0, (uint32_t)(L - 2)});
    if (cfg.feature_map == MMFHE_FEATURE_LEARNED) {
        p->keys.push_back(mmfhe_const_key{MMFHE_CONST_NOTCH_B, 0, 0, (uint32_t)(L - 2)});
        p->keys.push_back(mmfhe_const_key{MMFHE_CONST_FEAT_A, 0, 0, (uint32_t)(L - 3)});
    }
    // FC1 reads the features: level L - 3 - (the feature map's depth)
    const int lf = L - 3 - gesture_feature_depth(cfg);
    for (int k = 0; k < W; k++) p->keys.push_back(mmfhe_const_key{MMFHE_CONST_FCW, 0, (uint32_t)k, (uint32_t)lf});
    p->keys.push_back(mmfhe_const_key{MMFHE_CONST_FCB, 0, 0, (uint32_t)(lf - 1)});
    for (int l = 1; l <= 2; l++)
        for (int k : fc_present(cfg, l))
            p->keys.push_back(mmfhe_const_key{MMFHE_CONST_FCW, (uint32_t)l, (uint32_t)k, (uint32_t)(lf - 2 * l)});
    for (int b = 1; b < p->n1_k3; b++) rots.insert(norm_rot(c, b));
    for (int f = 1; f < p->fpc; f <<= 1) rots.insert(norm_rot(c, f * p->ard_pad));
    for (int b = 1; b < p->n1_fc; b++) rots.insert(norm_rot(c, b));
    for (int g = 1; g < W / p->n1_fc; g++) rots.insert(norm_rot(c, g * p->n1_fc));
    for (int s = W; s < p->ard_pad; s <<= 1) rots.insert(norm_rot(c, s));
    rots.erase(0);
    p->rotations.assign(rots.begin(), rots.end());
    p->n_in = cfg.complex_slots ? p->pairs : 2 * p->pairs;
    p->out_levels = {lf - 5};
    p->consts.resize(p->keys.size());
    for (size_t i = 0; i < p->keys.size(); i++) p->index[key_of(p->keys[i])] = (int)i;
    return p.release();
}

// Scale of FC1's rescaled output for inputs encrypted at scale `s0`: the
// evaluator's scale arithmetic step by step (products multiply scales, a
// rescale at level l divides by q_l, constants carry q_l).
// Scale of the notched power (after K3, K1 and the notch).
static double gesture_notch_scale(const Context &c, double s0) {
    auto q = [&](int l) { return (double)c.primes[l]; };
    const int L = c.L;
    double s = s0 * q(L) / q(L);
    s = s * s / q(L - 1);
    return s * q(L - 2) / q(L - 2);
}

static double gesture_fc1_scale(const Context &c, const mmfhe_circuit_config &cfg) {
    auto q = [&](int l) { return (double)c.primes[l]; };
    const int L = c.L;
    const double p = gesture_notch_scale(c, cfg.input_scale);
    if (cfg.feature_map == MMFHE_FEATURE_LEARNED) {
        const double f = p * p / q(L - 3);         // (notched p) x (b p + a)
        return f * q(L - 4) / q(L - 4);
    }
    double w = p * p / q(L - 3);
    w = w * w / q(L - 4);
    const double f = p * w / q(L - 5);
    return f * q(L - 6) / q(L - 6);
}

static Plan *create_fc_plan(Context &c, const mmfhe_circuit_config &cfg) {
    std::unique_ptr<Plan> p(new Plan());
    p->ctx = &c;
    p->cfg = cfg;
    const int D = (int)cfg.bins, L = (int)cfg.taps;
    std::tie(p->n1_dft, p->n2_dft) = bsgs_split(D);
    for (int l = 0; l < L; l++) {
        const int lv = c.L - 2 * l;   // a dense layer and a square take one level each
        for (int k : fc_present(cfg, l)) p->keys.push_back(mmfhe_const_key{MMFHE_CONST_FCW, (uint32_t)l, (uint32_t)k, (uint32_t)lv});
    }
    std::set<int32_t> rots;
    for (int b = 1; b < p->n1_dft; b++) rots.insert(norm_rot(c, b));
    for (int g = 1; g < p->n2_dft; g++) rots.insert(norm_rot(c, g * p->n1_dft));
    rots.erase(0);
    p->rotations.assign(rots.begin(), rots.end());
    p->n_in = 1;
    p->out_levels = {c.L - 2 * L + 1};
    p->consts.resize(p->keys.size());
    for (size_t i = 0; i < p->keys.size(); i++) p->index[key_of(p->keys[i])] = (int)i;
    return p.release();
}

// The library's FP64 design of the per-frame chain's scalar constants, in the
// order of mmfhe_plan_set_scalars.
static std::vector<double> per_frame_scalars(const Plan &p) {
    const mmfhe_circuit_config &cfg = p.cfg;
    const int F = (int)cfg.frames;
    const double fs = cfg.fs_mhz / 1000.0;
    std::vector<double> out;
    for (int b = 0; b < 2; b++) {
        std::vector<double> h = fir_bandpass((int)cfg.taps, cfg.band_lo_mhz[b] / 1000.0, cfg.band_hi_mhz[b] / 1000.0, fs);
        out.insert(out.end(), h.begin(), h.end());
    }
    for (int b = 0; b < 2; b++) {
        const double gain = cfg.dft_gain[b] / 3.0;
        for (int k : p.bands[b]) {
            for (int t = 1; t < F; t++) out.push_back(gain * hann(t, F) * std::cos(2 * M_PI * k * t / F));
            for (int t = 1; t < F; t++) out.push_back(-gain * hann(t, F) * std::sin(2 * M_PI * k * t / F));
        }
    }
    for (int b = 0; b < 2; b++)
        for (int k : p.bands[b]) out.push_back(k * fs / F);
    return out;
}

static Plan *create_per_frame_plan(Context &c, const mmfhe_circuit_config &cfg) {
    std::unique_ptr<Plan> p(new Plan());
    p->ctx = &c;
    p->cfg = cfg;
    const int L = c.L, F = (int)cfg.frames;
    for (int b = 0; b < 2; b++) {
        p->bands[b] = band_bins(F, (int)cfg.fs_mhz, (int)cfg.band_lo_mhz[b], (int)cfg.band_hi_mhz[b]);
        if (p->bands[b].empty()) throw Error(MMFHE_ERR_BAD_ARG, "empty frequency band");
    }
    p->span[0] = next_pow2((int)cfg.bins);
    p->keys.push_back(mmfhe_const_key{MMFHE_CONST_IDX, 0, 0, (uint32_t)(L - 2)});
    p->keys.push_back(mmfhe_const_key{MMFHE_CONST_ONE, 0, 0, (uint32_t)(L - 2)});
    for (int i = 0; (1 << i) < p->span[0]; i++) p->rotations.push_back(norm_rot(c, 1 << i));
    std::sort(p->rotations.begin(), p->rotations.end());
    p->n_in = 4 * F;
    p->out_levels = {L - 3, L - 3, L - 11, L - 11, L - 11, L - 11};
    p->scalars = per_frame_scalars(*p);
    p->consts.resize(p->keys.size());
    for (size_t i = 0; i < p->keys.size(); i++) p->index[key_of(p->keys[i])] = (int)i;
    return p.release();
}

Plan *create_plan(Context &c, const mmfhe_circuit_config &cfg_in) {
    mmfhe_circuit_config cfg = cfg_in;
    if (cfg.kind == MMFHE_CIRCUIT_GESTURE) {
        check_cfg(c, cfg);
        return create_gesture_plan(c, cfg);
    }
    if (is_vital(cfg) && cfg.dft_gain[0] == 0.0 && cfg.dft_gain[1] == 0.0) {
        // default public spectral gains (median DFT magnitude ~0.5 on the synthetic workload)
        cfg.dft_gain[0] = cfg.taylor_order == 3 ? 30.0 : 1.5;
        cfg.dft_gain[1] = cfg.taylor_order == 3 ? 1.0 : 0.2;
    }
    check_cfg(c, cfg);
    if (cfg.kind == MMFHE_CIRCUIT_FC) return create_fc_plan(c, cfg);
    if (cfg.kind == MMFHE_CIRCUIT_VITAL_PER_FRAME) return create_per_frame_plan(c, cfg);
    std::unique_ptr<Plan> p(new Plan());
    p->ctx = &c;
    p->cfg = cfg;
    p->f_pad = next_pow2((int)cfg.frames);
    p->r_c = (int)(c.n / 2) / p->f_pad;
    p->groups = ((int)cfg.bins + p->r_c - 1) / p->r_c;
    std::tie(p->n1_fir, p->n2_fir) = bsgs_split((int)cfg.taps);
    std::tie(p->n1_dft, p->n2_dft) = bsgs_split(p->f_pad);
    const int L = c.L, Fp = p->f_pad, F = (int)cfg.frames;
    auto add = [&](uint32_t tag, uint32_t band, uint32_t idx, int level) {
        if (level < 0) throw Error(MMFHE_ERR_BAD_ARG, "not enough levels in the parameter set for this circuit");
        p->keys.push_back(mmfhe_const_key{tag, band, idx, (uint32_t)level});
    };
    std::set<int32_t> rots;
    auto rot = [&](int32_t k) { rots.insert(norm_rot(c, k)); };
    if (cfg.kind == MMFHE_CIRCUIT_FIR_DFT) {
        if (L < 2) throw Error(MMFHE_ERR_BAD_ARG, "FIR+DFT needs at least 3 Q primes");
        for (uint32_t k = 0; k < cfg.taps; k++) add(MMFHE_CONST_FIR, 0, k, L);
        std::set<int> present;
        for (int d = 0; d < F; d++)
            for (int n = 0; n < F; n++) present.insert(((n - d) % Fp + Fp) % Fp);
        p->dft_deltas[0].assign(present.begin(), present.end());
        for (uint32_t tag : {MMFHE_CONST_DFT_C, MMFHE_CONST_DFT_S, MMFHE_CONST_DFT_MS})
            for (int d : p->dft_deltas[0]) add(tag, 0, d, L - 1);
        for (int b = 1; b < p->n1_fir; b++) rot(-b * p->r_c);
        for (int g = 1; g < p->n2_fir; g++) rot(-g * p->n1_fir * p->r_c);
        for (int d : p->dft_deltas[0]) {
            if (d % p->n1_dft) rot((d % p->n1_dft) * p->r_c);
            if (d / p->n1_dft) rot((d / p->n1_dft) * p->n1_dft * p->r_c);
        }
        p->n_in = 2 * p->groups;
        for (int g = 0; g < p->groups; g++) {
            p->out_levels.push_back(L - 2);
            p->out_levels.push_back(L - 2);
        }
    } else {
        const int lv_side = L - 3, lv_fir = L - 3;
        const int lv_dphi = cfg.taylor_order == 3 ? L - 7 : L - 5;
        const int lv_final = lv_dphi - 3;
        if (lv_final < 1) throw Error(MMFHE_ERR_BAD_ARG, "not enough levels for the vital chain");
        p->lv_side = lv_side;
        p->lv_fir = lv_fir;
        p->lv_dphi = lv_dphi;
        p->lv_final = lv_final;
        // side branch: the first-block mask at L - 1, index / one vectors at the packed block starts
        add(MMFHE_CONST_PMASK, 0, 0, L - 1);
        add(MMFHE_CONST_IDX, 0, 0, lv_side);
        add(MMFHE_CONST_ONE, 0, 0, lv_side);
        for (int b = 0; b < 2; b++)
            for (uint32_t k = 0; k < cfg.taps; k++) add(MMFHE_CONST_FIR, b, k, lv_fir);
        // from the FIR on, band b lives in bin slot b of every frame
        if (p->r_c < 2) throw Error(MMFHE_ERR_BAD_ARG, "the vital chain needs two bin slots per frame");
        std::set<int> present;
        for (int b = 0; b < 2; b++) {
            p->bands[b] = band_bins(F, (int)cfg.fs_mhz, (int)cfg.band_lo_mhz[b], (int)cfg.band_hi_mhz[b]);
            if (p->bands[b].empty()) throw Error(MMFHE_ERR_BAD_ARG, "empty frequency band");
            if (p->bands[b].back() >= Fp / 2) throw Error(MMFHE_ERR_BAD_ARG, "band beyond half the padded window");
            // rows: Re X_k at k, Im X_k at k + F_pad/2
            for (int k : p->bands[b])
                for (int t = 0; t < F; t++)
                    for (int row : {k, k + Fp / 2}) present.insert(((t - row) % Fp + Fp) % Fp);
            p->span[b] = next_pow2(p->bands[b].back() + 1);
        }
        p->dft_deltas[0].assign(present.begin(), present.end());
        for (int d : p->dft_deltas[0]) add(MMFHE_CONST_DRE, 0, d, lv_dphi);
        for (uint32_t b = 0; b < 2; b++) {   // one weight pair per band
            add(MMFHE_CONST_FW, b, 0, lv_final);
            add(MMFHE_CONST_FONE, b, 0, lv_final);
        }
        for (int i = 0; (1 << i) < Fp; i++) rot(p->r_c << i);
        for (int i = 0; (1 << i) < p->r_c; i++) rot(1 << i);
        for (int b = 0; b < p->n1_fir; b++) {
            rot(-b * p->r_c);
            rot(-b * p->r_c - 1);
        }
        for (int g = 1; g < p->n2_fir; g++) rot(-g * p->n1_fir * p->r_c);
        rot(-p->r_c);
        for (int d : p->dft_deltas[0]) {
            if (d % p->n1_dft) rot((d % p->n1_dft) * p->r_c);
            if (d / p->n1_dft) rot((d / p->n1_dft) * p->n1_dft * p->r_c);
        }
        for (int i = 0; (1 << i) < std::max(p->span[0], p->span[1]); i++) rot(p->r_c << i);
        rot((Fp / 2) * p->r_c);
        rot(1);
        for (int b = 0; b < 2; b++) rot(-p->span[b] * p->r_c);   // den beside num in a band's sums
        if (cfg.complex_slots) rots.insert(MMFHE_ROT_CONJ);
        p->n_in = (cfg.complex_slots ? 2 : 4) * p->groups;
        // the side branch (num_r, den_r), band RR, band HR
        p->out_levels = {lv_side - 1, lv_final - 1, lv_final - 1};
    }
    rots.erase(0);
    p->rotations.assign(rots.begin(), rots.end());
    p->consts.resize(p->keys.size());
    for (size_t i = 0; i < p->keys.size(); i++) p->index[key_of(p->keys[i])] = (int)i;
    return p.release();
}

const PtDev &plan_const(const Plan &p, uint32_t tag, uint32_t band, uint32_t idx) {
    auto it = p.index.find(((uint64_t)tag << 48) | ((uint64_t)band << 40) | idx);
    if (it == p.index.end()) throw Error(MMFHE_ERR_NOT_FOUND, "plan constant missing");
    const PtDev &pt = p.consts[it->second];
    if (!pt.buf.get()) throw Error(MMFHE_ERR_NOT_FOUND, "plan constant " + std::to_string(it->second) + " not set");
    return pt;
}

// The vital chain's FIR and DFT products are double-hoisted: their diagonals
// multiply baby steps over the extended basis Q_l * P and are kept there.
static bool const_is_qp(const Plan &p, const mmfhe_const_key &k) {
    return p.cfg.kind == MMFHE_CIRCUIT_VITAL && (k.tag == MMFHE_CONST_FIR || k.tag == MMFHE_CONST_DRE);
}

void plan_set_const(Plan &p, uint32_t i, const uint64_t *words_host_or_dev, cudaStream_t st) {
    Context &c = *p.ctx;
    if (i >= p.keys.size()) throw Error(MMFHE_ERR_BAD_ARG, "constant index out of range");
    // the context pool reuses a freed buffer at once, which is safe only in
    // stream order; evaluations may run on a caller's stream, so wait for
    // all device work before this set-up step allocates from the pool
    CK(cudaDeviceSynchronize());
    const int level = (int)p.keys[i].level;
    if (const_is_qp(p, p.keys[i])) {
        p.consts[i] = pt_qp_from_coeffs(c, words_host_or_dev, level, (double)c.primes[level], st);
        return;
    }
    PtDev pt = pt_new(c, level, (double)c.primes[level]);
    CK(cudaMemcpyAsync(pt.buf.get(), words_host_or_dev, (size_t)(level + 1) * c.n * 8, cudaMemcpyDefault, st));
    ntt_q_blocks(c, pt.buf.get(), 1, level + 1, false, st);
    pt_to_mont(c, pt, st);   // plan constants are kept in Montgomery form
    p.consts[i] = std::move(pt);
}

// slot vector of constant k with the library's own FP64 design
static std::vector<double> const_slots(const Plan &p, const mmfhe_const_key &k) {
    const Context &c = *p.ctx;
    const mmfhe_circuit_config &cfg = p.cfg;
    const int n = (int)c.n / 2, Rc = p.r_c, Fp = p.f_pad, F = (int)cfg.frames;
    std::vector<double> v(n, 0.0), out(n, 0.0);
    auto slot = [&](int t, int r) { return t * Rc + r; };
    auto prerot = [&](int g, int n1, int stride) {
        // D' = Rot(D, -g n1 stride): out[j] = v[(j - g n1 stride) mod n]
        long long sh = (long long)g * n1 * stride;
        for (int j = 0; j < n; j++) out[j] = v[(int)((((j - sh) % n) + n) % n)];
        return out;
    };
    const double fs = cfg.fs_mhz / 1000.0;
    switch (k.tag) {
    case MMFHE_CONST_IDX:
    case MMFHE_CONST_ONE:
        if (cfg.kind == MMFHE_CIRCUIT_VITAL_PER_FRAME) {   // bin r in slot r
            for (int r = 0; r < (int)cfg.bins; r++) v[r] = k.tag == MMFHE_CONST_IDX ? (double)r : 1.0;
            return v;
        }
        {   // group g's bins at the start of its packed block (-g mod G')
            const int Gp = next_pow2(p.groups), blk = Fp / Gp;
            for (int g = 0; g < p.groups; g++)
                for (int r = 0; r < Rc; r++) {
                    const int gb = g * Rc + r;
                    if (gb < (int)cfg.bins)
                        v[slot(((Gp - g) % Gp) * blk, r)] = k.tag == MMFHE_CONST_IDX ? (double)gb : 1.0;
                }
        }
        return v;
    case MMFHE_CONST_PMASK: {   // the first F_pad / G' frames of every bin slot
        const int blk = Fp / next_pow2(p.groups);
        for (int t = 0; t < blk; t++)
            for (int r = 0; r < Rc; r++) v[slot(t, r)] = 1.0;
        return v;
    }
    case MMFHE_CONST_FIR: {
        int b = (int)k.band, kk = (int)k.index;
        std::vector<double> h = fir_bandpass((int)cfg.taps, cfg.band_lo_mhz[b] / 1000.0, cfg.band_hi_mhz[b] / 1000.0, fs);
        // VITAL: band b's taps act in bin slot b; FIR_DFT: every bin
        const int r0 = cfg.kind == MMFHE_CIRCUIT_VITAL ? b : 0, r1 = cfg.kind == MMFHE_CIRCUIT_VITAL ? b + 1 : Rc;
        for (int t = kk; t < F; t++)
            for (int r = r0; r < r1; r++) v[slot(t, r)] = h[kk];
        return prerot(kk / p.n1_fir, p.n1_fir, -Rc);
    }
    case MMFHE_CONST_DRE: {
        // the DFT rows of both bands: Re X_k in row k, Im X_k in row k + F_pad/2,
        // band b in bin slot b; diag_d[row] = M[row, row + d]
        const int d = (int)k.index;
        for (int b = 0; b < 2; b++) {
            // the phase signal carries 3 dphi (third order); with complex slots 6i dphi or 2i dphi
            const double gain = cfg.complex_slots ? cfg.dft_gain[b] / (cfg.taylor_order == 3 ? 6.0 : 2.0)
                                                  : cfg.dft_gain[b] * (cfg.taylor_order == 3 ? 1.0 / 3.0 : 1.0);
            for (int kk : p.bands[b]) {
                for (int part = 0; part < 2; part++) {
                    const int row = kk + part * (Fp / 2);
                    const int t = (row + d) % Fp;
                    if (t < F) {
                        double ang = 2 * M_PI * kk * t / F;
                        v[slot(row, b)] = gain * hann(t, F) * (part == 0 ? std::cos(ang) : -std::sin(ang));
                    }
                }
            }
        }
        return prerot(d / p.n1_dft, p.n1_dft, Rc);
    }
    case MMFHE_CONST_DFT_C:
    case MMFHE_CONST_DFT_S:
    case MMFHE_CONST_DFT_MS: {
        int d = (int)k.index, D = F;
        for (int row = 0; row < D; row++) {
            int col = (row + d) % Fp;
            if (col >= D) continue;
            int sig = (row + D / 2) % D;
            double ang = -2 * M_PI * sig * col / D;
            double w = hann(col, D);
            double val = k.tag == MMFHE_CONST_DFT_C ? w * std::cos(ang) : w * std::sin(ang);
            if (k.tag == MMFHE_CONST_DFT_MS) val = -val;
            for (int r = 0; r < Rc; r++) v[slot(row, r)] = val;
        }
        return prerot(d / p.n1_dft, p.n1_dft, Rc);
    }
    case MMFHE_CONST_GDFT_C:
    case MMFHE_CONST_GDFT_S:
    case MMFHE_CONST_GDFT_MS:
    case MMFHE_CONST_GDFT_W: {   // GDFT_W: the real part (C); plan_encode_consts adds S as the imaginary part
        // block-diagonal I (x) M of Eq. K3 on every active slot:
        // diag_delta[s] = M[i][i + delta], i = s mod D
        const int D = (int)cfg.chirps, delta = (int)k.index - D;
        const int ard = (int)(cfg.antennas * cfg.bins * cfg.chirps);
        for (int s = 0; s < n; s++) {
            const int i = s % D, j = i + delta;
            if (j < 0 || j >= D || s % p.ard_pad >= ard) continue;
            const int sig = (i + D / 2) % D;
            const double ang = -2 * M_PI * sig * j / D, w = hann(j, D);
            double val = (k.tag == MMFHE_CONST_GDFT_C || k.tag == MMFHE_CONST_GDFT_W) ? w * std::cos(ang)
                                                                                  : w * std::sin(ang);
            v[s] = k.tag == MMFHE_CONST_GDFT_MS ? -val : val;
        }
        return prerot(floor_div(delta, p.n1_k3), p.n1_k3, 1);
    }
    case MMFHE_CONST_NOTCH:
    case MMFHE_CONST_NOTCH_B: {
        // Eq. (notch mask): zero on Doppler bins floor(D/2) .. ceil(D/2); NOTCH_B: times b
        const int D = (int)cfg.chirps, ard = (int)(cfg.antennas * cfg.bins * cfg.chirps);
        const double g = k.tag == MMFHE_CONST_NOTCH_B ? cfg.feature_coef[1] : 1.0;
        for (int s = 0; s < n; s++) {
            const int d = s % D;
            v[s] = (s % p.ard_pad < ard && !(d >= D / 2 && d <= (D + 1) / 2)) ? g : 0.0;
        }
        return v;
    }
    case MMFHE_CONST_FEAT_A: {
        // a on every active slot (the notched product it joins is zero elsewhere)
        const int ard = (int)(cfg.antennas * cfg.bins * cfg.chirps);
        for (int s = 0; s < n; s++) v[s] = s % p.ard_pad < ard ? cfg.feature_coef[0] : 0.0;
        return v;
    }
    case MMFHE_CONST_FW:
    case MMFHE_CONST_FONE:
        // band k.band only: frequency k fs / F (or 1) at (k, band)
        for (int kk : p.bands[k.band]) v[slot(kk, (int)k.band)] = k.tag == MMFHE_CONST_FW ? kk * fs / F : 1.0;
        return v;
    }
    throw Error(MMFHE_ERR_BAD_ARG, "unknown constant tag");
}

void plan_encode_consts(Plan &p, cudaStream_t st) {
    Context &c = *p.ctx;
    // the context pool reuses a freed buffer at once, which is safe only in
    // stream order; evaluations may run on a caller's stream, so wait for
    // all device work before this set-up step allocates from the pool
    CK(cudaDeviceSynchronize());
    if (p.cfg.kind == MMFHE_CIRCUIT_FC)
        throw Error(MMFHE_ERR_BAD_ARG, "FC constants are learned weights: set them with mmfhe_plan_set_fc_layer");
    std::vector<uint64_t> words;
    for (size_t i = 0; i < p.keys.size(); i++) {
        const mmfhe_const_key &k = p.keys[i];
        if (k.tag == MMFHE_CONST_FCW || k.tag == MMFHE_CONST_FCB) continue;   // learned: set_fc_layer
        std::vector<double> v = const_slots(p, k), im;
        if (k.tag == MMFHE_CONST_GDFT_W) {   // complex W = C + i S
            mmfhe_const_key ks = k;
            ks.tag = MMFHE_CONST_GDFT_S;
            im = const_slots(p, ks);
        }
        words.assign((size_t)(k.level + 1) * c.n, 0);
        // a constant that is added (not multiplied) is encoded at the scale of its ciphertext
        const double scale = k.tag == MMFHE_CONST_FEAT_A ? gesture_notch_scale(c, p.cfg.input_scale)
                                                         : (double)c.primes[k.level];
        encode_slots(c.params, v.data(), scale, (int)k.level, words.data(), im.empty() ? nullptr : im.data());
        plan_set_const(p, (uint32_t)i, words.data(), st);
        CK(cudaStreamSynchronize(st));
    }
}

// ---------------------------------------------------------------------------
// circuit executors (all windows of the batch in every launch)
// ---------------------------------------------------------------------------
static CtB square_sum(Context &c, const Keys &k, const std::vector<const CtB *> &xs, cudaStream_t st) {
    TensorB t = tensor_new(c, xs[0]->B, xs[0]->level);
    for (size_t i = 0; i < xs.size(); i++) tensor_acc(c, t, *xs[i], *xs[i], 1, i == 0, st);
    return relin(c, k, t, st);
}

static std::vector<CtB> run_fir_dft(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in, cudaStream_t st) {
    const int Rc = p.r_c;
    std::vector<CtB> out;
    std::vector<int> all_fir(p.n1_fir), rot_fir(p.n1_fir);
    for (int b = 0; b < p.n1_fir; b++) { all_fir[b] = b; rot_fir[b] = -b * Rc; }
    BsgsTerm fir;
    for (uint32_t kk = 0; kk < p.cfg.taps; kk++) fir.diags.push_back({(int)kk, &plan_const(p, MMFHE_CONST_FIR, 0, kk)});
    fir.baby_idx = all_fir;
    std::vector<int> all_dft(p.n1_dft), rot_dft(p.n1_dft);
    for (int b = 0; b < p.n1_dft; b++) { all_dft[b] = b; rot_dft[b] = b * Rc; }
    for (int g = 0; g < p.groups; g++) {
        CtB vf[2];
        for (int part = 0; part < 2; part++) {
            std::vector<CtB> babies = rotate_hoisted(c, k, in[2 * g + part], rot_fir, st);
            BsgsTerm t = fir;
            t.baby = &babies;
            vf[part] = rescale(c, bsgs(c, k, {t}, p.n1_fir, -Rc, st), st);
        }
        std::vector<CtB> bre = rotate_hoisted(c, k, vf[0], rot_dft, st);
        std::vector<CtB> bim = rotate_hoisted(c, k, vf[1], rot_dft, st);
        auto term = [&](const std::vector<CtB> *bb, uint32_t tag) {
            BsgsTerm t;
            t.baby = bb;
            t.baby_idx = all_dft;
            for (int d : p.dft_deltas[0]) t.diags.push_back({d, &plan_const(p, tag, 0, d)});
            return t;
        };
        out.push_back(rescale(c, bsgs(c, k, {term(&bre, MMFHE_CONST_DFT_C), term(&bim, MMFHE_CONST_DFT_MS)}, p.n1_dft, Rc, st), st));
        out.push_back(rescale(c, bsgs(c, k, {term(&bre, MMFHE_CONST_DFT_S), term(&bim, MMFHE_CONST_DFT_C)}, p.n1_dft, Rc, st), st));
    }
    return out;
}

// The vital chain on complex slots (z = Re + i Im per group and stream):
// |z|^2 = z conj(z); K4 gives Z = I + i Q; one FIR product per band filters
// both parts; K7 w = Z conj(Z at t-1) = x + i y, the phase signal
// w^3 - conj(w^3) = 2i Im(w^3) (third order) or w - conj(w) (first); K3,
// |X|^2, sharpening and the sums as in the split chain.
// Baby sets of the vital FIR product on x: RR taps on Rot(x, -b R_c) (output
// in bin slot 0), HR taps on Rot(x, -b R_c - 1) (slot 1).
static std::vector<BsgsSet> fir_sets(const Plan &p, const CtB &x) {
    std::vector<BsgsSet> sets(2);
    for (int band = 0; band < 2; band++) {
        sets[band].x = &x;
        sets[band].offset = -band;
        for (uint32_t kk = 0; kk < p.cfg.taps; kk++)
            sets[band].diags.push_back({(int)kk, &plan_const(p, MMFHE_CONST_FIR, band, kk)});
    }
    return sets;
}

// The narrowband DFT's single baby set on dphi: Rot(dphi, b R_c).
static std::vector<BsgsSet> dft_sets(const Plan &p, const CtB &dphi) {
    std::vector<BsgsSet> sets(1);
    sets[0].x = &dphi;
    for (int d : p.dft_deltas[0]) sets[0].diags.push_back({d, &plan_const(p, MMFHE_CONST_DRE, 0, d)});
    return sets;
}

// K1 -> K2 on the G groups' energies ps (frame-major, stride r_c): each
// group's frame sums over t + j F_pad / G' (G' = G rounded up to a power of
// two) by a rotate-and-sum, the first frame block kept by a mask, the groups
// packed into one ciphertext by a rotation tree (group g lands in block
// -g mod G'), one rotate-and-sum over a block, w = E^2 once, and
// rotate-and-sums over the bins and then over the blocks.  Returns
// one ciphertext holding num_r in slot 0 and den_r in slot r_c (den's
// products moved one frame on before the sums).
static CtB side_branch(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &ps, cudaStream_t st) {
    const int Rc = p.r_c, Gp = next_pow2(p.groups), blk = p.f_pad / Gp;
    const PtDev &mask = plan_const(p, MMFHE_CONST_PMASK, 0, 0);
    std::vector<CtB> parts;
    for (CtB &x : ps) {
        CtB s = rotsum(c, k, x, blk * Rc, (uint32_t)Gp, st);
        x = CtB();
        CtB t = ct_new(c, s.B, s.level, s.scale * mask.scale);
        ct_mul_plain(c, t, s, mask, false, st);
        parts.push_back(rescale(c, t, st));
    }
    parts.resize(Gp);   // missing groups: empty (level -1)
    for (int j = 0; parts.size() > 1; j++) {
        std::vector<CtB> nxt;
        for (size_t a = 0; a < parts.size(); a += 2) {
            CtB &x = parts[a], &y = parts[a + 1];
            if (y.level < 0) {
                nxt.push_back(std::move(x));
            } else if (x.level < 0) {
                nxt.push_back(rotate(c, k, y, (blk << j) * Rc, st));
            } else {
                nxt.push_back(rotate_add(c, k, y, (blk << j) * Rc, x, st));
            }
        }
        parts = std::move(nxt);
    }
    CtB E = rotsum(c, k, parts[0], Rc, (uint32_t)blk, st);
    parts.clear();
    CtB w = rescale(c, square_sum(c, k, {&E}, st), st);
    CtB t[2];
    for (int i = 0; i < 2; i++) {
        const PtDev &pt = plan_const(p, i == 0 ? MMFHE_CONST_IDX : MMFHE_CONST_ONE, 0, 0);
        CtB x = ct_new(c, w.B, w.level, w.scale * pt.scale);
        ct_mul_plain(c, x, w, pt, false, st);
        t[i] = rescale(c, x, st);
    }
    // den's terms one frame on, beside num's in one ciphertext
    CtB r = rotate_add(c, k, t[1], -Rc, t[0], st);
    r = rotsum(c, k, r, 1, (uint32_t)Rc, st);
    return rotsum(c, k, r, blk * Rc, (uint32_t)Gp, st);
}

// Weighted frequency average of both bands from the sharpened powers S (band
// b in bin slot b): per band, its own weight and one masks, den's products
// moved span_b frames on beside num's, and one rotate-and-sum over the span,
// so each band's sums leave in a ciphertext of their own (a band far stronger
// than the other cannot overflow the other's sums at the last level): num_b
// in slot b, den_b in slot span_b r_c + b.  Returns the RR and HR ciphertexts.
static std::vector<CtB> band_sums(Context &c, const Plan &p, const Keys &k, const CtB &S, cudaStream_t st) {
    const int B = S.B;
    std::vector<CtB> out;
    for (int b = 0; b < 2; b++) {
        CtB t[2];
        for (int i = 0; i < 2; i++) {
            const PtDev &pt = plan_const(p, i == 0 ? MMFHE_CONST_FW : MMFHE_CONST_FONE, (uint32_t)b, 0);
            CtB x = ct_new(c, B, S.level, S.scale * pt.scale);
            ct_mul_plain(c, x, S, pt, false, st);
            t[i] = rescale(c, x, st);
        }
        CtB r = rotate_add(c, k, t[1], -p.span[b] * p.r_c, t[0], st);
        out.push_back(rotsum(c, k, r, p.r_c, (uint32_t)p.span[b], st));
    }
    return out;
}

static std::vector<CtB> run_vital_complex(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in,
                                          cudaStream_t st) {
    const int G = p.groups, Rc = p.r_c;
    const int B = in[0].B;
    auto abs2 = [&](const CtB &z) {
        CtB zc = rotate(c, k, z, MMFHE_ROT_CONJ, st);
        TensorB t = tensor_new(c, B, z.level);
        tensor_acc(c, t, z, zc, 1, true, st);
        return rescale(c, relin(c, k, t, st), st);
    };
    // ---- side branch: K1, K2 ----
    std::vector<CtB> ps;
    for (int g = 0; g < G; g++) ps.push_back(abs2(in[g]));
    CtB side = side_branch(c, p, k, ps, st);
    // ---- K4: Z = sum_r m z ----
    std::vector<CtB> m;
    for (int g = 0; g < G; g++) {
        CtB pp = abs2(in[G + g]);
        m.push_back(rescale(c, square_sum(c, k, {&pp}, st), st));
    }
    const int lv = m[0].level;
    TensorB t4 = tensor_new(c, B, lv);
    for (int g = 0; g < G; g++) {
        CtB x = ct_drop(c, in[G + g], lv, st);
        tensor_acc(c, t4, m[g], x, 1, g == 0, st);
    }
    m.clear();
    CtB Z = rotsum(c, k, rescale(c, relin(c, k, t4, st), st), 1, (uint32_t)Rc, st);
    // ---- K5: both bands in one double-hoisted product (RR in bin slot 0, HR in slot 1) ----
    CtB Zf = rescale(c, bsgs_dh(c, k, fir_sets(p, Z), p.n1_fir, -Rc, st), st);
    // ---- K7: w = Zf conj(Zf at t-1) ----
    CtB zpc = rotate(c, k, rotate(c, k, Zf, -Rc, st), MMFHE_ROT_CONJ, st);
    TensorB tw = tensor_new(c, B, Zf.level);
    tensor_acc(c, tw, Zf, zpc, 1, true, st);
    CtB wc = rescale(c, relin(c, k, tw, st), st);
    CtB dphi;
    {
        CtB top;
        if (p.cfg.taylor_order == 3) {
            CtB w2 = rescale(c, square_sum(c, k, {&wc}, st), st);
            CtB wd = ct_drop(c, wc, w2.level, st);
            TensorB t3 = tensor_new(c, B, w2.level);
            tensor_acc(c, t3, wd, w2, 1, true, st);
            top = rescale(c, relin(c, k, t3, st), st);
        } else {
            top = std::move(wc);
        }
        CtB topc = rotate(c, k, top, MMFHE_ROT_CONJ, st);
        dphi = ct_new(c, B, top.level, top.scale);
        ct_addsub(c, dphi, top, topc, true, st);
    }
    // ---- K3, |X|^2 (negated by the i), sharpen, weighted frequency average ----
    CtB X = rescale(c, bsgs_dh(c, k, dft_sets(p, dphi), p.n1_dft, Rc, st), st);
    CtB pw = rescale(c, square_sum(c, k, {&X}, st), st);
    CtB merged = rotate_add(c, k, pw, (p.f_pad / 2) * Rc, pw, st);
    CtB S = rescale(c, square_sum(c, k, {&merged}, st), st);
    std::vector<CtB> out;
    out.push_back(std::move(side));
    for (CtB &x : band_sums(c, p, k, S, st)) out.push_back(std::move(x));
    return out;
}

static std::vector<CtB> run_vital(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in, cudaStream_t st) {
    if (p.cfg.complex_slots) return run_vital_complex(c, p, k, in, st);
    const int G = p.groups, Rc = p.r_c;
    const int B = in[0].B;
    // ---- side branch: K1, K2 ----
    std::vector<CtB> ps;
    for (int g = 0; g < G; g++) ps.push_back(rescale(c, square_sum(c, k, {&in[2 * g], &in[2 * g + 1]}, st), st));
    CtB side = side_branch(c, p, k, ps, st);
    // ---- K4 soft I/Q ----
    std::vector<CtB> m;
    for (int g = 0; g < G; g++) {
        const CtB &re = in[2 * G + 2 * g], &im = in[2 * G + 2 * g + 1];
        CtB pp = rescale(c, square_sum(c, k, {&re, &im}, st), st);
        m.push_back(rescale(c, square_sum(c, k, {&pp}, st), st));
    }
    const int lv = m[0].level;
    CtB iq[2];
    for (int part = 0; part < 2; part++) {
        TensorB t = tensor_new(c, B, lv);
        for (int g = 0; g < G; g++) {
            CtB x = ct_drop(c, in[2 * G + 2 * g + part], lv, st);
            tensor_acc(c, t, m[g], x, 1, g == 0, st);
        }
        iq[part] = rotsum(c, k, rescale(c, relin(c, k, t, st), st), 1, (uint32_t)Rc, st);
    }
    m.clear();
    // ---- K5 FIR of both bands in one double-hoisted BSGS product per part:
    // baby steps share one ModUp, unshifted for RR (bin slot 0), one slot on
    // for HR (slot 1) ----
    CtB filt[2];
    for (int part = 0; part < 2; part++)
        filt[part] = rescale(c, bsgs_dh(c, k, fir_sets(p, iq[part]), p.n1_fir, -Rc, st), st);
    // ---- K7, both bands slot by slot ----
    const CtB &If = filt[0], &Qf = filt[1];
    CtB If1 = rotate(c, k, If, -Rc, st);
    CtB Qf1 = rotate(c, k, Qf, -Rc, st);
    TensorB ty = tensor_new(c, B, If.level);
    tensor_acc(c, ty, Qf, If1, 1, true, st);
    tensor_acc(c, ty, If, Qf1, -1, false, st);
    CtB y = rescale(c, relin(c, k, ty, st), st);
    TensorB tx = tensor_new(c, B, If.level);
    tensor_acc(c, tx, If, If1, 1, true, st);
    tensor_acc(c, tx, Qf, Qf1, 1, false, st);
    CtB x = rescale(c, relin(c, k, tx, st), st);
    CtB dphi;
    if (p.cfg.taylor_order == 3) {
        TensorB tu = tensor_new(c, B, x.level);
        tensor_acc(c, tu, x, x, 3, true, st);
        tensor_acc(c, tu, y, y, -1, false, st);
        CtB u = rescale(c, relin(c, k, tu, st), st);
        CtB yd = ct_drop(c, y, u.level, st);
        TensorB tp = tensor_new(c, B, u.level);
        tensor_acc(c, tp, yd, u, 1, true, st);
        dphi = rescale(c, relin(c, k, tp, st), st);
    } else {
        dphi = std::move(y);
    }
    // ---- K3 narrowband DFT (both bands, each in its bin slot), |X|^2 ----
    CtB X = rescale(c, bsgs_dh(c, k, dft_sets(p, dphi), p.n1_dft, Rc, st), st);
    CtB pw = rescale(c, square_sum(c, k, {&X}, st), st);
    // Re^2 at k, Im^2 at k + F_pad/2: one rotation adds them
    CtB merged = rotate_add(c, k, pw, (p.f_pad / 2) * Rc, pw, st);
    // ---- sharpen, weighted frequency average (RR in slot 0, HR in slot 1) ----
    CtB S = rescale(c, square_sum(c, k, {&merged}, st), st);
    std::vector<CtB> out;
    out.push_back(std::move(side));
    for (CtB &x : band_sums(c, p, k, S, st)) out.push_back(std::move(x));
    return out;
}

// Polynomial network: per layer, hoisted baby rotations of the input, the
// BSGS product with the layer's diagonals, a rescale, and a square (relin,
// rescale) after every layer but the last.
static std::vector<CtB> run_fc(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in, cudaStream_t st) {
    const int L = (int)p.cfg.taps, n1 = p.n1_dft;
    std::vector<int32_t> rot(n1);
    std::vector<int> idx(n1);
    for (int b = 0; b < n1; b++) rot[b] = idx[b] = b;
    CtB x = std::move(in[0]);
    for (int l = 0; l < L; l++) {
        std::vector<CtB> babies = rotate_hoisted(c, k, x, rot, st);
        BsgsTerm t;
        t.baby = &babies;
        t.baby_idx = idx;
        for (int d : fc_present(p.cfg, l)) t.diags.push_back({d, &plan_const(p, MMFHE_CONST_FCW, (uint32_t)l, (uint32_t)d)});
        CtB y = rescale(c, bsgs(c, k, {t}, n1, 1, st), st);
        if (l < L - 1) {
            TensorB sq = tensor_new(c, y.B, y.level);
            tensor_acc(c, sq, y, y, 1, true, st);
            y = rescale(c, relin(c, k, sq, st), st);
        }
        x = std::move(y);
    }
    std::vector<CtB> out;
    out.push_back(std::move(x));
    return out;
}

static void encode_and_set(Plan &p, const mmfhe_const_key &key0, const std::vector<double> &v, double scale) {
    Context &c = *p.ctx;
    const auto it = p.index.find(key_of(key0));
    if (it == p.index.end()) throw Error(MMFHE_ERR_NOT_FOUND, "plan constant missing");
    const mmfhe_const_key &key = p.keys[it->second];
    std::vector<uint64_t> words((size_t)(key.level + 1) * c.n, 0);
    encode_slots(c.params, v.data(), scale > 0 ? scale : (double)c.primes[key.level], (int)key.level, words.data());
    plan_set_const(p, (uint32_t)it->second, words.data(), 0);
    CK(cudaStreamSynchronize(0));
}

// Gesture FC layers.  Layer 0: W is fc_width x (A R D + 1); extended
// diagonal k: diag_k[s] = W[s mod w][(s + k) mod ARD_pad] (zero on padding
// columns and on row w-1), pre-rotated by its giant step; the bias vector
// b[s mod w] with 1 in slot w-1, encoded at the scale of FC1's rescaled
// output.  Layers 1, 2: w x w as in FC plans.
static void gesture_set_fc_layer(Plan &p, uint32_t layer, const double *W) {
    Context &c = *p.ctx;
    const mmfhe_circuit_config &cfg = p.cfg;
    const int w = (int)cfg.fc_width, n1 = p.n1_fc, slots = (int)c.n / 2;
    const int ard = (int)(cfg.antennas * cfg.bins * cfg.chirps);
    std::vector<double> v(slots), r(slots);
    auto prerot = [&](int g) {
        const int sh = g * n1;
        for (int j = 0; j < slots; j++) r[j] = v[((j - sh) % slots + slots) % slots];
    };
    if (layer == 0) {
        const size_t ld = (size_t)ard + 1;
        for (int k = 0; k < w; k++) {
            for (int s = 0; s < slots; s++) {
                const int col = (s + k) % p.ard_pad, row = s % w;
                v[s] = (col < ard && row != w - 1) ? W[(size_t)row * ld + col] : 0.0;
            }
            prerot(k / n1);
            encode_and_set(p, mmfhe_const_key{MMFHE_CONST_FCW, 0, (uint32_t)k, 0}, r, 0.0);
        }
        for (int s = 0; s < slots; s++) v[s] = s % w == w - 1 ? 1.0 : W[(size_t)(s % w) * ld + ard];
        encode_and_set(p, mmfhe_const_key{MMFHE_CONST_FCB, 0, 0, 0}, v, gesture_fc1_scale(c, cfg));
        return;
    }
    for (int k : fc_present(cfg, (int)layer)) {
        for (int s = 0; s < slots; s++) v[s] = W[(size_t)(s % w) * w + ((s % w) + k) % w];
        prerot(k / n1);
        encode_and_set(p, mmfhe_const_key{MMFHE_CONST_FCW, layer, (uint32_t)k, 0}, r, 0.0);
    }
}

// Gesture chain: in[0] / in[1] = Re / Im of every pair of every window
// (batch B pairs, window-major).
// The gesture chain's feature stage runs on at most this many ciphertext
// pairs at a time (whole windows): its hoisted Doppler baby steps and key
// switches hold about 0.17 GB of scratch per pair at N = 2^15, so a batch of
// 16 windows (480 pairs) in one piece would need about 80 GB.  Every
// operation of the stage acts on each ciphertext alone, so the chunking
// changes no word.
constexpr int GESTURE_PAIRS_PER_CHUNK = 128;

static CtB gesture_features(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in, cudaStream_t st);

static std::vector<CtB> run_gesture(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in,
                                    cudaStream_t st) {
    const mmfhe_circuit_config &cfg = p.cfg;
    const int W = (int)cfg.fc_width;
    const int B = in[0].B / p.pairs;
    const int wchunk = std::max(1, GESTURE_PAIRS_PER_CHUNK / p.pairs);
    CtB feat;
    if (B <= wchunk) {
        feat = gesture_features(c, p, k, in, st);
    } else {
        // the windows' pairs are window-major: a chunk of whole windows is a contiguous slice
        for (int b0 = 0; b0 < B; b0 += wchunk) {
            const int nb = std::min(wchunk, B - b0);
            std::vector<CtB> part;
            for (const CtB &x : in) part.push_back(ct_slice(c, x, b0 * p.pairs, nb * p.pairs, st));
            CtB f = gesture_features(c, p, k, part, st);
            if (b0 == 0) feat = ct_new(c, B, f.level, f.scale);
            ct_place(c, feat, b0, f, st);
        }
        in.clear();
    }
    const int n1 = p.n1_fc;
    std::vector<int32_t> rb(n1);
    std::vector<int> idx(n1);
    for (int b = 0; b < n1; b++) rb[b] = idx[b] = b;
    CtB x = std::move(feat);
    for (int l = 0; l < 3; l++) {
        std::vector<CtB> babies = rotate_hoisted(c, k, x, rb, st);
        BsgsTerm t;
        t.baby = &babies;
        t.baby_idx = idx;
        if (l == 0)
            for (int d = 0; d < W; d++) t.diags.push_back({d, &plan_const(p, MMFHE_CONST_FCW, 0, (uint32_t)d)});
        else
            for (int d : fc_present(cfg, l)) t.diags.push_back({d, &plan_const(p, MMFHE_CONST_FCW, (uint32_t)l, (uint32_t)d)});
        CtB y = rescale(c, bsgs(c, k, {t}, n1, 1, st), st);
        babies.clear();
        if (l == 0)
            y = add_plain(c, rotsum(c, k, y, W, (uint32_t)(p.ard_pad / W), st), plan_const(p, MMFHE_CONST_FCB, 0, 0), st);
        if (l < 2) y = rescale(c, square_sum(c, k, {&y}, st), st);
        x = std::move(y);
    }
    std::vector<CtB> out;
    out.push_back(std::move(x));
    return out;
}

// K3 -> K1 -> K6 -> soft power -> weighting on every pair of the given
// windows (in: Re and Im of every pair, or one complex-slot ciphertext per
// pair, window-major), then the accumulation over each window's frames: one
// feature ciphertext per window.
static CtB gesture_features(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in, cudaStream_t st) {
    const mmfhe_circuit_config &cfg = p.cfg;
    const int D = (int)cfg.chirps;
    CtB feat;
    {
        std::vector<int32_t> rb(p.n1_k3);
        std::vector<int> idx(p.n1_k3);
        for (int b = 0; b < p.n1_k3; b++) rb[b] = idx[b] = b;
        CtB pw;
        if (cfg.complex_slots) {
            // K3 on Re + i Im: one product with the complex W; K1 |d|^2 = d conj(d)
            std::vector<CtB> bz = rotate_hoisted(c, k, in[0], rb, st);
            in.clear();
            BsgsTerm tz;
            tz.baby = &bz;
            tz.baby_idx = idx;
            for (int delta = -(D - 1); delta < D; delta++)
                tz.diags.push_back({delta, &plan_const(p, MMFHE_CONST_GDFT_W, 0, (uint32_t)(delta + D))});
            CtB d = rescale(c, bsgs(c, k, {tz}, p.n1_k3, 1, st), st);
            bz.clear();
            CtB dc = rotate(c, k, d, MMFHE_ROT_CONJ, st);
            TensorB tt = tensor_new(c, d.B, d.level);
            tensor_acc(c, tt, d, dc, 1, true, st);
            pw = rescale(c, relin(c, k, tt, st), st);
        } else {
            // K3: d_re = C re - S im, d_im = S re + C im (Eq. K3), one BSGS each
            std::vector<CtB> bre = rotate_hoisted(c, k, in[0], rb, st);
            std::vector<CtB> bim = rotate_hoisted(c, k, in[1], rb, st);
            in.clear();
            BsgsTerm t[4];
            for (int i = 0; i < 4; i++) {
                t[i].baby = i % 2 == 0 ? &bre : &bim;
                t[i].baby_idx = idx;
            }
            for (int delta = -(D - 1); delta < D; delta++) {
                const uint32_t ix = (uint32_t)(delta + D);
                t[0].diags.push_back({delta, &plan_const(p, MMFHE_CONST_GDFT_C, 0, ix)});
                t[1].diags.push_back({delta, &plan_const(p, MMFHE_CONST_GDFT_MS, 0, ix)});
                t[2].diags.push_back({delta, &plan_const(p, MMFHE_CONST_GDFT_S, 0, ix)});
                t[3].diags.push_back({delta, &plan_const(p, MMFHE_CONST_GDFT_C, 0, ix)});
            }
            CtB dre = rescale(c, bsgs(c, k, {t[0], t[1]}, p.n1_k3, 1, st), st);
            CtB dim = rescale(c, bsgs(c, k, {t[2], t[3]}, p.n1_k3, 1, st), st);
            bre.clear();
            bim.clear();
            pw = rescale(c, square_sum(c, k, {&dre, &dim}, st), st);                  // K1
        }
        CtB pm = ct_new(c, pw.B, pw.level, pw.scale);
        ct_mul_plain(c, pm, pw, plan_const(p, MMFHE_CONST_NOTCH, 0, 0), false, st);   // K6
        CtB pn = rescale(c, pm, st);
        if (cfg.feature_map == MMFHE_FEATURE_LEARNED) {
            // learned map a p + b p^2 = (notched p) x (b notched p + a): one level
            const PtDev &nb = plan_const(p, MMFHE_CONST_NOTCH_B, 0, 0);
            CtB pbm = ct_new(c, pw.B, pw.level, pw.scale * nb.scale);
            ct_mul_plain(c, pbm, pw, nb, false, st);
            CtB pba = add_plain(c, rescale(c, pbm, st), plan_const(p, MMFHE_CONST_FEAT_A, 0, 0), st);
            TensorB tf = tensor_new(c, pn.B, pn.level);
            tensor_acc(c, tf, pn, pba, 1, true, st);
            CtB f = rescale(c, relin(c, k, tf, st), st);
            return rotsum(c, k, group_sum(c, f, p.pairs, st), p.ard_pad, (uint32_t)p.fpc, st);
        }
        CtB w2 = rescale(c, square_sum(c, k, {&pn}, st), st);                     // w = p^4
        CtB w4 = rescale(c, square_sum(c, k, {&w2}, st), st);
        CtB pd = ct_drop(c, pn, w4.level, st);
        TensorB tw = tensor_new(c, w4.B, w4.level);
        tensor_acc(c, tw, pd, w4, 1, true, st);
        CtB f = rescale(c, relin(c, k, tw, st), st);                          // p x w
        feat = rotsum(c, k, group_sum(c, f, p.pairs, st), p.ard_pad, (uint32_t)p.fpc, st);
    }
    return feat;
}

void plan_set_fc_layer(Plan &p, uint32_t layer, const double *W) {
    Context &c = *p.ctx;
    if (p.cfg.kind == MMFHE_CIRCUIT_GESTURE) {
        if (layer > 2) throw Error(MMFHE_ERR_BAD_ARG, "layer out of range");
        return gesture_set_fc_layer(p, layer, W);
    }
    if (p.cfg.kind != MMFHE_CIRCUIT_FC) throw Error(MMFHE_ERR_BAD_ARG, "not an FC plan");
    if (layer >= p.cfg.taps) throw Error(MMFHE_ERR_BAD_ARG, "layer out of range");
    const int D = (int)p.cfg.bins, n1 = p.n1_dft, slots = (int)c.n / 2;
    std::vector<double> v(slots), r(slots);
    std::vector<uint64_t> words;
    for (int k : fc_present(p.cfg, (int)layer)) {
        // diag_k[j] = W[j mod D][(j mod D + k) mod D], pre-rotated by the giant step
        for (int j = 0; j < slots; j++) v[j] = W[(size_t)(j % D) * D + ((j % D) + k) % D];
        const int sh = (k / n1) * n1;   // Rot(v, -sh)[j] = v[j - sh]
        for (int j = 0; j < slots; j++) r[j] = v[((j - sh) % slots + slots) % slots];
        const auto it = p.index.find(key_of(mmfhe_const_key{MMFHE_CONST_FCW, layer, (uint32_t)k, 0}));
        const mmfhe_const_key &key = p.keys[it->second];
        words.assign((size_t)(key.level + 1) * c.n, 0);
        encode_slots(c.params, r.data(), (double)c.primes[key.level], (int)key.level, words.data());
        plan_set_const(p, (uint32_t)it->second, words.data(), 0);
        CK(cudaStreamSynchronize(0));
    }
}

// Per-frame packing: in = stream 1 (Re_t, Im_t) for t < F, then stream 2.
// Sums over bins are rotate-and-sums (result in slot 0); sums over frames and
// the FIR / DFT are scalar linear combinations of frame ciphertexts.
static std::vector<CtB> run_vital_per_frame(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in,
                                            cudaStream_t st) {
    const mmfhe_circuit_config &cfg = p.cfg;
    const int F = (int)cfg.frames, T = (int)cfg.taps;
    const uint32_t span = (uint32_t)p.span[0];
    const std::vector<double> &sc = p.scalars;
    size_t si = 0;
    std::vector<double> taps[2];
    for (int b = 0; b < 2; b++) taps[b].assign(sc.begin() + si, sc.begin() + si + T), si += T;
    std::vector<std::vector<double>> cre[2], cim[2];
    for (int b = 0; b < 2; b++)
        for (size_t kk = 0; kk < p.bands[b].size(); kk++) {
            cre[b].emplace_back(sc.begin() + si, sc.begin() + si + F - 1), si += F - 1;
            cim[b].emplace_back(sc.begin() + si, sc.begin() + si + F - 1), si += F - 1;
        }
    std::vector<double> fhz[2];
    for (int b = 0; b < 2; b++) fhz[b].assign(sc.begin() + si, sc.begin() + si + p.bands[b].size()), si += p.bands[b].size();
    auto qs = [&](int level) { return (double)c.primes[level]; };
    // side branch: K1 energy summed over frames; K2 w = E^2; index / ones; rotate-sum over bins
    CtB E;
    for (int t = 0; t < F; t++) {
        CtB pt = rescale(c, square_sum(c, k, {&in[2 * t], &in[2 * t + 1]}, st), st);
        if (t == 0) {
            E = std::move(pt);
        } else {
            CtB e2 = ct_new(c, E.B, E.level, E.scale);
            ct_addsub(c, e2, E, pt, false, st);
            E = std::move(e2);
        }
    }
    CtB w = rescale(c, square_sum(c, k, {&E}, st), st);
    CtB num = ct_new(c, w.B, w.level, w.scale), den = ct_new(c, w.B, w.level, w.scale);
    ct_mul_plain(c, num, w, plan_const(p, MMFHE_CONST_IDX, 0, 0), false, st);
    ct_mul_plain(c, den, w, plan_const(p, MMFHE_CONST_ONE, 0, 0), false, st);
    std::vector<CtB> outs;
    outs.push_back(rotsum(c, k, rescale(c, num, st), 1, span, st));
    outs.push_back(rotsum(c, k, rescale(c, den, st), 1, span, st));
    // K4 soft I/Q per frame
    std::vector<CtB> I, Q;
    for (int t = 0; t < F; t++) {
        const CtB &re = in[2 * F + 2 * t], &im = in[2 * F + 2 * t + 1];
        CtB pp = rescale(c, square_sum(c, k, {&re, &im}, st), st);
        CtB m = rescale(c, square_sum(c, k, {&pp}, st), st);
        for (int part = 0; part < 2; part++) {
            CtB x = ct_drop(c, part == 0 ? re : im, m.level, st);
            TensorB tt = tensor_new(c, m.B, m.level);
            tensor_acc(c, tt, m, x, 1, true, st);
            (part == 0 ? I : Q).push_back(rotsum(c, k, rescale(c, relin(c, k, tt, st), st), 1, span, st));
        }
    }
    std::map<int, CtB> S;
    for (int b = 0; b < 2; b++) {
        // K5 causal FIR over frames
        std::vector<CtB> If, Qf;
        for (int t = 0; t < F; t++) {
            for (int part = 0; part < 2; part++) {
                const std::vector<CtB> &X = part == 0 ? I : Q;
                std::vector<std::pair<const CtB *, double>> terms;
                for (int kk = 0; kk < T && t - kk >= 0; kk++) terms.push_back({&X[t - kk], taps[b][kk]});
                (part == 0 ? If : Qf).push_back(rescale(c, lincomb(c, terms, qs(X[0].level), st), st));
            }
        }
        // K7 third order, frames t >= 1 (dphi[0] = 0)
        std::vector<CtB> dphi(F);
        for (int t = 1; t < F; t++) {
            TensorB ty = tensor_new(c, If[t].B, If[t].level);
            tensor_acc(c, ty, Qf[t], If[t - 1], 1, true, st);
            tensor_acc(c, ty, If[t], Qf[t - 1], -1, false, st);
            CtB y = rescale(c, relin(c, k, ty, st), st);
            TensorB tx = tensor_new(c, If[t].B, If[t].level);
            tensor_acc(c, tx, If[t], If[t - 1], 1, true, st);
            tensor_acc(c, tx, Qf[t], Qf[t - 1], 1, false, st);
            CtB x = rescale(c, relin(c, k, tx, st), st);
            TensorB tu = tensor_new(c, x.B, x.level);
            tensor_acc(c, tu, x, x, 3, true, st);
            tensor_acc(c, tu, y, y, -1, false, st);
            CtB u = rescale(c, relin(c, k, tu, st), st);
            CtB yd = ct_drop(c, y, u.level, st);
            TensorB tp = tensor_new(c, u.B, u.level);
            tensor_acc(c, tp, yd, u, 1, true, st);
            dphi[t] = rescale(c, relin(c, k, tp, st), st);
        }
        // K3 narrowband DFT per bin, |X|^2, square (bands are disjoint in k)
        for (size_t kk = 0; kk < p.bands[b].size(); kk++) {
            std::vector<std::pair<const CtB *, double>> tre, tim;
            for (int t = 1; t < F; t++) {
                tre.push_back({&dphi[t], cre[b][kk][t - 1]});
                tim.push_back({&dphi[t], cim[b][kk][t - 1]});
            }
            const double s = qs(dphi[1].level);
            CtB xr = rescale(c, lincomb(c, tre, s, st), st);
            CtB xi = rescale(c, lincomb(c, tim, s, st), st);
            CtB pk = rescale(c, square_sum(c, k, {&xr, &xi}, st), st);
            S[p.bands[b][kk]] = rescale(c, square_sum(c, k, {&pk}, st), st);
        }
    }
    for (int b = 0; b < 2; b++) {
        std::vector<std::pair<const CtB *, double>> tn, td;
        for (size_t kk = 0; kk < p.bands[b].size(); kk++) {
            tn.push_back({&S[p.bands[b][kk]], fhz[b][kk]});
            td.push_back({&S[p.bands[b][kk]], 1.0});
        }
        const double s = qs(S[p.bands[b][0]].level);
        outs.push_back(rescale(c, lincomb(c, tn, s, st), st));
        outs.push_back(rescale(c, lincomb(c, td, s, st), st));
    }
    return outs;
}

void plan_set_scalars(Plan &p, const double *v, size_t n) {
    if (p.cfg.kind != MMFHE_CIRCUIT_VITAL_PER_FRAME) throw Error(MMFHE_ERR_BAD_ARG, "only per-frame plans hold scalars");
    if (n != p.scalars.size()) throw Error(MMFHE_ERR_BAD_ARG, "wrong number of scalars");
    p.scalars.assign(v, v + n);
}

std::vector<CtB> run_plan(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in, cudaStream_t st) {
    if (p.cfg.kind == MMFHE_CIRCUIT_FC) return run_fc(c, p, k, in, st);
    if (p.cfg.kind == MMFHE_CIRCUIT_GESTURE) return run_gesture(c, p, k, in, st);
    if (p.cfg.kind == MMFHE_CIRCUIT_VITAL_PER_FRAME) return run_vital_per_frame(c, p, k, in, st);
    if (p.cfg.kind == MMFHE_CIRCUIT_FIR_DFT) return run_fir_dft(c, p, k, in, st);
    return run_vital(c, p, k, in, st);
}

}  // namespace mmfhe
