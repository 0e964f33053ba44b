/*
 * CPU oracle for the state-vector hot path.  TEST INFRASTRUCTURE ONLY: the tests,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs use it; the
 * library never links, loads or calls it.
 *
 * Plain, slow, complex128 code written from the paper's definitions.  It shares no
 * code with the CUDA library.  Amplitudes are stored interleaved (re, im) as doubles.
 * Qubit t is bit t of the amplitude index (little-endian), fixed by Eq. 3
 * (|psi'> = (I_{2^{n-t-1}} (x) U (x) I_{2^t}) |psi>, so qubit t has stride 2^t).
 *
 * Every loop is a plain loop over amplitudes; the outer loops carry an OpenMP
 * pragma so that the oracle finishes on large inputs, nothing else.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Apply one k-qubit gate U (2^k x 2^k, row-major, interleaved complex) to psi.
 *
 * Definition (Eq. 2 for k = 1, Eq. 3 in general, Eq. 4's gate = matrix + targets):
 *   psi'[i] = sum_c U[loc(i)][c] * psi[i with target bits replaced by c],
 *   loc(i)  = sum_j bit(i, targets[j]) * 2^j.
 * Evaluated group by group: every index i whose target bits are all zero is the base
 * of one group of 2^k amplitudes, and each group is an independent 2^k-vector
 * multiplied by U.  Targets may be given in any order; targets[j] is local bit j.
 */
int orc_apply(double *psi, int n, int k, const int *targets, const double *U) {
    if (k < 1 || k > 10 || k > n) return 1;
    uint64_t tmask = 0;
    for (int j = 0; j < k; ++j) {
        if (targets[j] < 0 || targets[j] >= n) return 1;
        if (tmask & (1ULL << targets[j])) return 1;
        tmask |= 1ULL << targets[j];
    }
    const uint64_t N = 1ULL << n;
    const int d = 1 << k;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)N; ++i) {
        if ((uint64_t)i & tmask) continue;       /* not a group base */
        double vr[1024], vi[1024];
        uint64_t idx[1024];
        for (int c = 0; c < d; ++c) {
            uint64_t off = 0;
            for (int j = 0; j < k; ++j)
                if ((c >> j) & 1) off |= 1ULL << targets[j];
            idx[c] = (uint64_t)i | off;
            vr[c] = psi[2 * idx[c]];
            vi[c] = psi[2 * idx[c] + 1];
        }
        for (int r = 0; r < d; ++r) {
            double ar = 0.0, ai = 0.0;
            for (int c = 0; c < d; ++c) {
                double ur = U[2 * (r * d + c)], ui = U[2 * (r * d + c) + 1];
                ar += ur * vr[c] - ui * vi[c];
                ai += ur * vi[c] + ui * vr[c];
            }
            psi[2 * idx[r]] = ar;
            psi[2 * idx[r] + 1] = ai;
        }
    }
    return 0;
}

/* sum_k |alpha_k|^2 (Eq. 1's normalisation). */
double orc_norm(const double *psi, int n) {
    const uint64_t N = 1ULL << n;
    double s = 0.0;
    int64_t i;
#pragma omp parallel for reduction(+:s) schedule(static)
    for (i = 0; i < (int64_t)N; ++i)
        s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    return s;
}

/* Z-basis probabilities p_k = |alpha_k|^2. */
void orc_probs(const double *psi, int n, double *p) {
    const uint64_t N = 1ULL << n;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)N; ++i)
        p[i] = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
}

static int popcount64(uint64_t x) {
    int c = 0;
    while (x) { c += (int)(x & 1); x >>= 1; }
    return c;
}

/*
 * <psi| P |psi> for the Pauli string P with X-part xmask and Z-part zmask
 * (qubit q carries X if only x_q, Z if only z_q, Y if both).  With Y = i X Z,
 *   P |k> = i^{|x & z|} (-1)^{popcount(k & z)} |k ^ x>,
 * so <psi|P|psi> = sum_k conj(psi[k ^ x]) i^{|x & z|} (-1)^{popcount(k & z)} psi[k].
 */
void orc_expect_pauli(const double *psi, int n, uint64_t xmask, uint64_t zmask,
                      double *out_re, double *out_im) {
    const uint64_t N = 1ULL << n;
    double sr = 0.0, si = 0.0;
    int64_t i;
#pragma omp parallel for reduction(+:sr,si) schedule(static)
    for (i = 0; i < (int64_t)N; ++i) {
        uint64_t k = (uint64_t)i, kx = k ^ xmask;
        double ar = psi[2 * k], ai = psi[2 * k + 1];
        double br = psi[2 * kx], bi = -psi[2 * kx + 1];          /* conj(psi[k^x]) */
        double pr = br * ar - bi * ai, pi = br * ai + bi * ar;
        if (popcount64(k & zmask) & 1) { pr = -pr; pi = -pi; }
        sr += pr;
        si += pi;
    }
    /* multiply by i^{|x&z|} */
    int y = popcount64(xmask & zmask) & 3;
    double rr = sr, ri = si;
    for (int t = 0; t < y; ++t) { double tmp = rr; rr = -ri; ri = tmp; }
    *out_re = rr;
    *out_im = ri;
}

/* <a|b> = sum_k conj(a_k) b_k. */
void orc_inner(const double *a, const double *b, int n, double *out_re, double *out_im) {
    const uint64_t N = 1ULL << n;
    double sr = 0.0, si = 0.0;
    int64_t i;
#pragma omp parallel for reduction(+:sr,si) schedule(static)
    for (i = 0; i < (int64_t)N; ++i) {
        double ar = a[2 * i], ai = -a[2 * i + 1];
        double br = b[2 * i], bi = b[2 * i + 1];
        sr += ar * br - ai * bi;
        si += ar * bi + ai * br;
    }
    *out_re = sr;
    *out_im = si;
}

/* |x>: all amplitudes zero except alpha_x = 1. */
void orc_set_basis(double *psi, int n, uint64_t x) {
    memset(psi, 0, sizeof(double) * 2 * (1ULL << n));
    psi[2 * x] = 1.0;
}
