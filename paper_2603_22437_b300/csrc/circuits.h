// Plans and circuit executors.
#pragma once
#include <map>
#include <vector>

#include "internal.h"

namespace mmfhe {

struct Plan {
    Context *ctx = nullptr;
    mmfhe_circuit_config cfg{};
    int f_pad = 0, r_c = 0, groups = 0;
    int n1_fir = 0, n2_fir = 0, n1_dft = 0, n2_dft = 0;
    int lv_side = -1, lv_fir = -1, lv_dphi = -1, lv_final = -1;
    std::vector<int> bands[2];
    std::vector<int> dft_deltas[2];
    int span[2] = {0, 0};
    std::vector<mmfhe_const_key> keys;          // constant order
    std::map<uint64_t, int> index;              // key -> position
    std::vector<PtDev> consts;                  // evaluation domain
    std::vector<int32_t> rotations;
    int n_in = 0;
    std::vector<int> out_levels;
    std::vector<double> scalars;                // per-frame chain: public scalar constants
    // gesture chain: padded frame size, frames per ciphertext, ciphertext
    // pairs per window, BSGS baby steps of the Doppler DFT and of the FC layers
    int ard_pad = 0, fpc = 0, pairs = 0, n1_k3 = 0, n1_fc = 0;
};

uint64_t key_of(const mmfhe_const_key &k);
std::vector<int> band_bins(int frames, int fs_mhz, int lo_mhz, int hi_mhz);
std::vector<double> fir_bandpass(int taps, double f_lo, double f_hi, double fs);
// imag (nullable): imaginary parts of complex slots.
void encode_slots(const mmfhe_params &p, const double *slots, double scale, int level, uint64_t *out,
                  const double *imag = nullptr);

Plan *create_plan(Context &c, const mmfhe_circuit_config &cfg);
const PtDev &plan_const(const Plan &p, uint32_t tag, uint32_t band, uint32_t idx);
void plan_set_const(Plan &p, uint32_t i, const uint64_t *words, cudaStream_t st);
void plan_encode_consts(Plan &p, cudaStream_t st);
void plan_set_fc_layer(Plan &p, uint32_t layer, const double *W);
void plan_set_scalars(Plan &p, const double *v, size_t n);
std::vector<int> fc_present(const mmfhe_circuit_config &cfg, int l);
std::vector<CtB> run_plan(Context &c, const Plan &p, const Keys &k, std::vector<CtB> &in, cudaStream_t st);

}  // namespace mmfhe
