// Host harness for the integer digit arithmetic of the complex128 tensor-core kernel
// (fixed_point.h): the same split, level sums and recombination the kernel performs for
// one group of 16 amplitudes, with the tensor-core accumulators replaced by exact
// integer sums.  Built and called by tests/test_fixed_point.py.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "../paper_2604_03816_gb300/csrc/fixed_point.h"

extern "C" {

long long fx_to_fixed(double x, unsigned emax) { return fxp::to_fixed(fxp::bits_of(x), emax); }

unsigned fx_exp_field(double x) { return fxp::exp_field(fxp::bits_of(x)); }

void fx_digits(long long x, int *d) {
    int t[fxp::DIGITS];
    fxp::digits(x, t);
    for (int i = 0; i < fxp::DIGITS; ++i) d[i] = t[i];
}

double fx_assemble(long long z, int p) { return fxp::assemble(z, p); }

double fx_assemble_words(long long z, int p) { return fxp::assemble_words(z, p); }

int fx_small_float_to_int(float v) { return fxp::small_float_to_int(v); }

double fx_combine_words(int i0, int i1, int i2, int i3, int i45, int p) {
    return fxp::combine_words(i0, i1, i2, i3, i45, p);
}

// The kernel's digit-pair words of the amplitude (re, im) on the grid of emax.
void fx_digit_pair_words(double re, double im, unsigned emax, unsigned *w) {
    const uint64_t br = fxp::bits_of(re), bi = fxp::bits_of(im);
    uint32_t rh, rl, ih, il, t[fxp::DIGITS];
    fxp::offset_fixed((uint32_t)(br >> 32), (uint32_t)br, emax, rh, rl);
    fxp::offset_fixed((uint32_t)(bi >> 32), (uint32_t)bi, emax, ih, il);
    fxp::digit_pair_words(rh, rl, ih, il, t);
    for (int i = 0; i < fxp::DIGITS; ++i) w[i] = t[i];
}

// a: 16 amplitudes (re, im); u: 16 x 16 row-major (re, im); out: 16 amplitudes.
// lmax[s] receives max |L_s| over the 32 outputs (s = 0..5).
void fx_group_apply(const double *a, const double *u, double *out, long long *lmax) {
    const int KD = 32;
    uint32_t emax = 1;
    for (int k = 0; k < KD; ++k) emax = std::max(emax, fxp::exp_field(fxp::bits_of(a[k])));
    // A digits through the kernel's word forms (pairs of components share a word)
    int ad[KD][6];
    for (int c = 0; c < 16; ++c) {
        unsigned w[6];
        fx_digit_pair_words(a[2 * c], a[2 * c + 1], emax, w);
        for (int i = 0; i < 6; ++i) {
            ad[2 * c][i] = (int)((w[i] & 0x3FFu)) - 256;
            ad[2 * c + 1][i] = (int)((w[i] >> 16) & 0x3FFu) - 256;
        }
    }
    double r[KD][KD], rmax = 0.0;
    for (int n = 0; n < KD; ++n)
        for (int kk = 0; kk < KD; ++kk) {
            const double re = u[2 * ((n >> 1) * 16 + (kk >> 1))];
            const double im = u[2 * ((n >> 1) * 16 + (kk >> 1)) + 1];
            r[n][kk] = ((n & 1) == (kk & 1)) ? re : ((n & 1) ? im : -im);
            rmax = std::max(rmax, std::fabs(r[n][kk]));
        }
    int eb = 0;
    std::frexp(rmax, &eb);
    const uint32_t ebias = (uint32_t)std::max(eb + 1022, 1);
    static int bd[KD][KD][6];
    for (int n = 0; n < KD; ++n)
        for (int kk = 0; kk < KD; ++kk) fxp::digits(fxp::to_fixed(fxp::bits_of(r[n][kk]), ebias), bd[n][kk]);
    for (int s = 0; s < 6; ++s) lmax[s] = 0;
    for (int n = 0; n < KD; ++n) {
        long long L[6] = {0, 0, 0, 0, 0, 0};
        for (int s = 0; s < 6; ++s)
            for (int i = 0; i <= s; ++i)
                for (int kk = 0; kk < KD; ++kk) L[s] += (long long)ad[kk][i] * bd[n][kk][s - i];
        for (int s = 0; s < 6; ++s) lmax[s] = std::max(lmax[s], L[s] < 0 ? -L[s] : L[s]);
        // the accumulators as FP32 values (exact for L0..L3), converted as the kernel does
        const float f0 = (float)L[0], f1 = (float)L[1], f2 = (float)L[2], f3 = (float)L[3];
        const float f45 = (float)((double)L[4] + (double)L[5] / 512.0);
        out[n] = fxp::combine_words(fxp::small_float_to_int(f0), fxp::small_float_to_int(f1),
                                    (int)std::nearbyint(f2), (int)std::nearbyint(f3),
                                    (int)std::nearbyint(16.0f * f45),
                                    (int)emax + ((int)ebias - 1022) - 1078);
    }
}
}
