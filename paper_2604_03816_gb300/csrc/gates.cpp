// Gate library (Eq. 4) and target sorting.  Host code, FP64.
//
// The canonical set G = {I, X, Y, Z, H, S, T, Rx, Ry, Rz, CNOT, CZ, SWAP, Toffoli, U3}
// with R_a(theta) = exp(-i theta A / 2); U3 in the OpenQASM 2 form; gates outside G are
// full unitaries: sqrt(P) = ((1+i) I + (1-i) P)/2 for P in {X, Y, W = (X+Y)/sqrt2},
// fSim(theta, phi), CP(phi).  Local bit j of a matrix belongs to targets[j].
#include <cmath>
#include <cstring>

#include "sv_internal.h"

namespace {

using svi::cplx;
const cplx I1(0.0, 1.0);

struct M {
    uint32_t k;
    cplx a[64];   // up to 8 x 8
    cplx &at(int r, int c) { return a[r * (1 << k) + c]; }
};

M eye(uint32_t k) {
    M m{k, {}};
    for (int i = 0; i < (1 << k); ++i) m.at(i, i) = 1.0;
    return m;
}

M m2(cplx a, cplx b, cplx c, cplx d) {
    M m{1, {}};
    m.a[0] = a; m.a[1] = b; m.a[2] = c; m.a[3] = d;
    return m;
}

M perm_swap(uint32_t k, int x, int y) {
    M m = eye(k);
    m.at(x, x) = 0; m.at(y, y) = 0; m.at(x, y) = 1; m.at(y, x) = 1;
    return m;
}

M sqrt_pauli(cplx p00, cplx p01, cplx p10, cplx p11) {
    const cplx a = (1.0 + I1) / 2.0, b = (1.0 - I1) / 2.0;
    return m2(a + b * p00, b * p01, b * p10, a + b * p11);
}

}  // namespace

extern "C" sv_status sv_gate_matrix(uint32_t kind, const double *params, uint32_t nparams,
                                    int dagger, double *u_out, uint32_t *k_out) {
    svi::clear_error();
    if (!u_out || !k_out) return svi::set_error(SV_ERR_ARG, "sv_gate_matrix: null output");
    static const int need[] = {0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 0, 0, 0, 0, 3, 0, 0, 0, 2, 1};
    if (kind > SV_GATE_UNITARY) return svi::set_error(SV_ERR_ARG, "sv_gate_matrix: unknown kind");
    if (kind == SV_GATE_UNITARY) {
        uint32_t k = 0;
        while (k <= SV_MAX_K && 2u * (1u << (2 * k)) != nparams) ++k;
        if (k == 0 || k > SV_MAX_K || !params)
            return svi::set_error(SV_ERR_ARG, "sv_gate_matrix: UNITARY needs 2*4^k params, 1<=k<=5");
        const int d = 1 << k;
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                const int src = dagger ? (c * d + r) : (r * d + c);
                u_out[2 * (r * d + c)] = params[2 * src];
                u_out[2 * (r * d + c) + 1] = dagger ? -params[2 * src + 1] : params[2 * src + 1];
            }
        *k_out = k;
        return SV_OK;
    }
    if ((int)nparams != need[kind] || (need[kind] && !params))
        return svi::set_error(SV_ERR_ARG, "sv_gate_matrix: wrong number of parameters");
    const double s2 = 1.0 / std::sqrt(2.0);
    const double th = nparams > 0 ? params[0] : 0.0;
    M m{1, {}};
    switch (kind) {
        case SV_GATE_I: m = eye(1); break;
        case SV_GATE_X: m = m2(0, 1, 1, 0); break;
        case SV_GATE_Y: m = m2(0, -I1, I1, 0); break;
        case SV_GATE_Z: m = m2(1, 0, 0, -1); break;
        case SV_GATE_H: m = m2(s2, s2, s2, -s2); break;
        case SV_GATE_S: m = m2(1, 0, 0, I1); break;
        case SV_GATE_T: m = m2(1, 0, 0, std::polar(1.0, M_PI / 4)); break;
        case SV_GATE_RX:   // cos(t/2) I - i sin(t/2) X
            m = m2(std::cos(th / 2), -I1 * std::sin(th / 2), -I1 * std::sin(th / 2), std::cos(th / 2));
            break;
        case SV_GATE_RY:
            m = m2(std::cos(th / 2), -std::sin(th / 2), std::sin(th / 2), std::cos(th / 2));
            break;
        case SV_GATE_RZ:
            m = m2(std::polar(1.0, -th / 2), 0, 0, std::polar(1.0, th / 2));
            break;
        case SV_GATE_U3: {
            const double t = params[0], p = params[1], l = params[2];
            m = m2(std::cos(t / 2), -std::polar(1.0, l) * std::sin(t / 2),
                   std::polar(1.0, p) * std::sin(t / 2), std::polar(1.0, p + l) * std::cos(t / 2));
            break;
        }
        case SV_GATE_SQRTX: m = sqrt_pauli(0, 1, 1, 0); break;
        case SV_GATE_SQRTY: m = sqrt_pauli(0, -I1, I1, 0); break;
        case SV_GATE_SQRTW: m = sqrt_pauli(0, s2 * (1.0 - I1), s2 * (1.0 + I1), 0); break;
        case SV_GATE_CNOT: m = perm_swap(2, 1, 3); break;    // local index c + 2 t
        case SV_GATE_CZ: m = eye(2); m.at(3, 3) = -1; break;
        case SV_GATE_SWAP: m = perm_swap(2, 1, 2); break;
        case SV_GATE_TOFFOLI: m = perm_swap(3, 3, 7); break;
        case SV_GATE_CP: m = eye(2); m.at(3, 3) = std::polar(1.0, th); break;
        case SV_GATE_FSIM: {
            const double t = params[0], p = params[1];
            m = eye(2);
            m.at(1, 1) = std::cos(t); m.at(2, 2) = std::cos(t);
            m.at(1, 2) = -I1 * std::sin(t); m.at(2, 1) = -I1 * std::sin(t);
            m.at(3, 3) = std::polar(1.0, -p);
            break;
        }
        default: return svi::set_error(SV_ERR_ARG, "sv_gate_matrix: unknown kind");
    }
    const int d = 1 << m.k;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            cplx v = dagger ? std::conj(m.at(c, r)) : m.at(r, c);
            u_out[2 * (r * d + c)] = v.real();
            u_out[2 * (r * d + c) + 1] = v.imag();
        }
    *k_out = m.k;
    return SV_OK;
}

namespace svi {

Gate sorted_gate(uint32_t k, const uint32_t *targets, const double *u) {
    Gate g;
    g.k = k;
    int order[SV_MAX_K];
    for (uint32_t j = 0; j < k; ++j) order[j] = (int)j;
    for (uint32_t a = 0; a < k; ++a)          // insertion sort by target
        for (uint32_t b = a + 1; b < k; ++b)
            if (targets[order[b]] < targets[order[a]]) std::swap(order[a], order[b]);
    for (uint32_t j = 0; j < k; ++j) g.t[j] = targets[order[j]];
    const int d = 1 << k;
    // new local bit j <- old local bit order[j]
    std::vector<int> old_of(d);
    for (int i = 0; i < d; ++i) {
        int o = 0;
        for (uint32_t j = 0; j < k; ++j)
            if ((i >> j) & 1) o |= 1 << order[j];
        old_of[i] = o;
    }
    g.u.resize((size_t)d * d);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            const int src = old_of[r] * d + old_of[c];
            g.u[(size_t)r * d + c] = cplx(u[2 * src], u[2 * src + 1]);
        }
    return g;
}

}  // namespace svi
