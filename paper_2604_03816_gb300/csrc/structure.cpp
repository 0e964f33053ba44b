// Exact structure of a gate matrix: control qubits, and a diagonal, monomial or dense
// remainder.  The paper's fusion densifies every gate and lists the unused structure and
// commutativity among its limits and future work (Sections 10-11).  The structure-aware
// passes rest on these definitions, taken on the stored FP64 entries, no tolerance:
//
// * local bit j is a control when U never changes bit j (U[r][c] = 0 whenever bit j of r
//   and of c differ) and U is the identity where bit j is 0 (U[r][c] = [r == c] there);
// * the reduced gate V is U restricted to the rows and columns whose control bits are
//   all 1, on the remaining targets in ascending order; then U = I outside that
//   subspace and V (x) I inside it;
// * V is diagonal (every off-diagonal entry 0), monomial (exactly one nonzero entry in
//   every row and every column) or dense; a 1 x 1 V equal to 1 makes U the identity.
#include "sv_internal.h"

namespace svi {

static bool is_control(const Gate &g, uint32_t j) {
    const uint32_t d = 1u << g.k, bj = 1u << j;
    const cplx zero(0.0, 0.0), one(1.0, 0.0);
    for (uint32_t r = 0; r < d; ++r)
        for (uint32_t c = 0; c < d; ++c) {
            const cplx u = g.u[(size_t)r * d + c];
            if ((r & bj) != (c & bj)) {
                if (u != zero) return false;
            } else if (!(r & bj) && u != (r == c ? one : zero)) {
                return false;
            }
        }
    return true;
}

Structure classify(const Gate &g) {
    Structure s;
    uint32_t keep[SV_MAX_K];
    uint32_t nk = 0;
    for (uint32_t j = 0; j < g.k; ++j) {
        if (is_control(g, j)) {
            s.ctrl |= 1u << j;
            s.ctrl_q[s.nctrl++] = g.t[j];
        } else {
            keep[nk++] = j;
        }
    }
    const uint32_t d = 1u << g.k, dv = 1u << nk;
    uint32_t idx[1 << SV_MAX_K];
    for (uint32_t a = 0; a < dv; ++a) {
        uint32_t x = s.ctrl;
        for (uint32_t i = 0; i < nk; ++i)
            if ((a >> i) & 1u) x |= 1u << keep[i];
        idx[a] = x;
    }
    s.v.k = nk;
    for (uint32_t i = 0; i < nk; ++i) s.v.t[i] = g.t[keep[i]];
    s.v.u.resize((size_t)dv * dv);
    for (uint32_t a = 0; a < dv; ++a)
        for (uint32_t b = 0; b < dv; ++b) s.v.u[(size_t)a * dv + b] = g.u[(size_t)idx[a] * d + idx[b]];

    const cplx zero(0.0, 0.0);
    if (dv == 1 && s.v.u[0] == cplx(1.0, 0.0)) {
        s.kind = SV_STRUCT_IDENTITY;
        return s;
    }
    bool diag = true;
    for (uint32_t a = 0; a < dv && diag; ++a)
        for (uint32_t b = 0; b < dv; ++b)
            if (a != b && s.v.u[(size_t)a * dv + b] != zero) {
                diag = false;
                break;
            }
    if (diag) {
        s.kind = SV_STRUCT_DIAGONAL;
        return s;
    }
    uint32_t colcount[1 << SV_MAX_K] = {0};
    bool mono = true;
    for (uint32_t a = 0; a < dv && mono; ++a) {
        uint32_t rowcount = 0;
        for (uint32_t b = 0; b < dv; ++b)
            if (s.v.u[(size_t)a * dv + b] != zero) {
                ++rowcount;
                ++colcount[b];
            }
        mono = rowcount == 1;
    }
    for (uint32_t b = 0; b < dv && mono; ++b) mono = colcount[b] == 1;
    s.kind = mono ? SV_STRUCT_MONOMIAL : SV_STRUCT_DENSE;
    return s;
}

}  // namespace svi
