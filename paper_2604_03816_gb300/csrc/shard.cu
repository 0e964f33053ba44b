// Global-qubit sharding of one state over 2^g processes (one GPU each).
//
// The paper keeps the whole state on one device and names its memory as the ceiling of
// the design (Section 10) and multi-device partitioning as future work (Section 11).
// Here the 2^n amplitudes are split by their top g index bits: rank r holds the 2^L
// amplitudes (L = n - g) whose top g bits equal r, as an ordinary L-qubit state.  A
// logical qubit sits at a physical bit position: positions below L are bits of the local
// index ("local"), position L + j is bit j of the rank ("global").  A gate whose
// targets are all local is an ordinary pass on every rank with its targets relabelled to
// their positions.  Before a gate touches a qubit at a global position, one exchange
// swaps it with a local position p: rank r (bit j of r = b) sends the half of its
// amplitudes whose local bit p is 1 - b to its partner r ^ 2^j and receives the partner's
// half into the same places.  Afterwards the qubit that was at p sits at global position j
// and the other one at p; nothing else moves.
//
// The planner (host) walks a fused schedule, chooses for every needed swap the local
// position whose qubit is used again latest (Belady's rule; ties to the highest position,
// whose half is contiguous), and at the end swaps every qubit back to its own position --
// global positions by exchanges, local ones by SWAP passes -- so that each rank ends with
// the amplitudes r 2^L .. (r + 1) 2^L - 1 in index order.  The exchanges themselves are
// done by the caller's transport (NCCL send/recv between processes); this file provides
// the pack and unpack kernels that move one half of a shard between the state and a
// contiguous staging buffer, chunk by chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <new>
#include <string>
#include <vector>

#include "sv_internal.h"

struct sv_shard_plan {
    uint32_t n = 0, g = 0, L = 0;
    struct Step {
        uint32_t kind = SV_SHARD_APPLY;
        uint32_t local_bit = 0, global_bit = 0;
        sv_circuit *seg = nullptr;
    };
    std::vector<Step> steps;
    uint64_t exchanges = 0, local_swaps = 0;
    ~sv_shard_plan() {
        for (Step &s : steps) delete s.seg;
    }
};

namespace svi {
namespace {

Gate relabel(const Gate &g, const uint32_t *phys) {
    uint32_t t[SV_MAX_K];
    for (uint32_t j = 0; j < g.k; ++j) t[j] = phys[g.t[j]];
    std::vector<double> u(2 * g.u.size());
    for (size_t i = 0; i < g.u.size(); ++i) {
        u[2 * i] = g.u[i].real();
        u[2 * i + 1] = g.u[i].imag();
    }
    return sorted_gate(g.k, t, u.data());
}

Gate swap_gate(uint32_t a, uint32_t b) {
    Gate s;
    s.k = 2;
    s.t[0] = std::min(a, b);
    s.t[1] = std::max(a, b);
    s.u.assign(16, cplx(0.0, 0.0));
    s.u[0] = s.u[1 * 4 + 2] = s.u[2 * 4 + 1] = s.u[15] = cplx(1.0, 0.0);
    return s;
}

struct Planner {
    uint32_t n, g, L;
    std::vector<uint32_t> phys, at;          // logical -> position, position -> logical
    sv_shard_plan *plan;
    std::vector<Gate> seg;

    void flush() {
        if (seg.empty()) return;
        sv_circuit *c = new sv_circuit();
        c->n = L;
        c->gates = std::move(seg);
        seg.clear();
        sv_shard_plan::Step st;
        st.kind = SV_SHARD_APPLY;
        st.seg = c;
        plan->steps.push_back(st);
    }
    void exchange(uint32_t p, uint32_t j) {          // local position p <-> global bit j
        flush();
        sv_shard_plan::Step st;
        st.kind = SV_SHARD_SWAP;
        st.local_bit = p;
        st.global_bit = j;
        plan->steps.push_back(st);
        const uint32_t a = at[p], b = at[L + j];
        at[p] = b;
        at[L + j] = a;
        phys[a] = L + j;
        phys[b] = p;
        ++plan->exchanges;
    }
};

}  // namespace
}  // namespace svi

using namespace svi;

extern "C" {

sv_status sv_shard_plan_create(const sv_circuit *c, uint32_t g, sv_dtype dtype, sv_shard_plan **out) {
    clear_error();
    if (!c || !out) return set_error(SV_ERR_ARG, "sv_shard_plan_create: null argument");
    *out = nullptr;
    if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "sv_shard_plan_create: bad dtype");
    if (g > 16 || g >= c->n) return set_error(SV_ERR_ARG, "sv_shard_plan_create: g must be below n and at most 16");
    const uint32_t L = c->n - g;
    // complex128 shards run width-5 gates as the input fused at width 4 (tensor cores)
    const std::vector<Gate> &gates = (dtype == SV_C128 && L >= 11) ? narrow_schedule(c) : c->gates;
    uint32_t kmax = 0;
    for (const Gate &gt : gates) kmax = std::max(kmax, gt.k);
    if (L < std::max(kmax, 2u))
        return set_error(SV_ERR_ARG, "sv_shard_plan_create: a shard of " + std::to_string(L) +
                                         " qubits cannot hold a gate of " + std::to_string(kmax) +
                                         " targets (needs n - g >= the widest gate and >= 2)");
    sv_shard_plan *plan = new (std::nothrow) sv_shard_plan();
    if (!plan) return set_error(SV_ERR_OOM, "sv_shard_plan_create: host allocation failed");
    try {
        plan->n = c->n;
        plan->g = g;
        plan->L = L;
        Planner P{c->n, g, L, {}, {}, plan, {}};
        P.phys.resize(c->n);
        P.at.resize(c->n);
        for (uint32_t q = 0; q < c->n; ++q) P.phys[q] = P.at[q] = q;
        // next use of each qubit: per qubit the gate indices that act on it, and a cursor
        std::vector<std::vector<uint32_t>> uses(c->n);
        for (uint32_t i = 0; i < gates.size(); ++i)
            for (uint32_t j = 0; j < gates[i].k; ++j) uses[gates[i].t[j]].push_back(i);
        std::vector<size_t> cur(c->n, 0);
        auto next_use = [&](uint32_t q, uint32_t i) -> uint64_t {
            while (cur[q] < uses[q].size() && uses[q][cur[q]] < i) ++cur[q];
            return cur[q] < uses[q].size() ? uses[q][cur[q]] : UINT64_MAX;
        };
        for (uint32_t i = 0; i < gates.size(); ++i) {
            const Gate &gt = gates[i];
            uint64_t tmask = 0;
            for (uint32_t j = 0; j < gt.k; ++j) tmask |= 1ull << gt.t[j];
            for (uint32_t j = 0; j < gt.k; ++j) {
                const uint32_t q = gt.t[j];
                if (P.phys[q] < L) continue;
                // evict the local qubit (not a target of this gate) used again latest
                uint32_t best = UINT32_MAX;
                uint64_t best_use = 0;
                for (uint32_t p = L; p-- > 0;) {
                    const uint32_t lq = P.at[p];
                    if (tmask & (1ull << lq)) continue;
                    const uint64_t u = next_use(lq, i);
                    if (best == UINT32_MAX || u > best_use) {
                        best = p;
                        best_use = u;
                    }
                }
                P.exchange(best, P.phys[q] - L);
            }
            P.seg.push_back(relabel(gt, P.phys.data()));
        }
        // every qubit back to its own position: global ones by exchanges ...
        for (uint32_t j = 0; j < g; ++j) {
            const uint32_t q = L + j;
            if (P.phys[q] == L + j) continue;
            if (P.phys[q] >= L) {            // at another global position: through a local one
                const uint32_t via = L - 1;
                P.exchange(via, P.phys[q] - L);
            }
            P.exchange(P.phys[q], j);
        }
        // ... and local ones by SWAP passes
        for (uint32_t p = 0; p < L; ++p)
            while (P.at[p] != p) {
                const uint32_t q = P.at[p];      // belongs at position q (< L)
                P.seg.push_back(swap_gate(p, q));
                std::swap(P.at[p], P.at[q]);
                P.phys[P.at[p]] = p;
                P.phys[P.at[q]] = q;
                ++plan->local_swaps;
            }
        P.flush();
    } catch (const std::bad_alloc &) {
        delete plan;
        return set_error(SV_ERR_OOM, "sv_shard_plan_create: host allocation failed");
    }
    *out = plan;
    return SV_OK;
}

sv_status sv_shard_plan_free(sv_shard_plan *p) {
    delete p;
    return SV_OK;
}

sv_status sv_shard_plan_info(const sv_shard_plan *p, size_t *nsteps, uint64_t *exchanges,
                             uint64_t *local_swaps) {
    clear_error();
    if (!p) return set_error(SV_ERR_ARG, "sv_shard_plan_info: null plan");
    if (nsteps) *nsteps = p->steps.size();
    if (exchanges) *exchanges = p->exchanges;
    if (local_swaps) *local_swaps = p->local_swaps;
    return SV_OK;
}

sv_status sv_shard_plan_step(const sv_shard_plan *p, size_t i, uint32_t *kind, uint32_t *local_bit,
                             uint32_t *global_bit, const sv_circuit **segment) {
    clear_error();
    if (!p || i >= p->steps.size()) return set_error(SV_ERR_ARG, "sv_shard_plan_step: bad index");
    const sv_shard_plan::Step &st = p->steps[i];
    if (kind) *kind = st.kind;
    if (local_bit) *local_bit = st.local_bit;
    if (global_bit) *global_bit = st.global_bit;
    if (segment) *segment = st.seg;
    return SV_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ pack / unpack

namespace svk {

// Element e of the half whose index bit `bit` is `val`: insert that bit into e.
__device__ __forceinline__ unsigned long long half_index(unsigned long long e, uint32_t bit, uint32_t val) {
    const unsigned long long lo = e & ((1ull << bit) - 1ull);
    return ((e >> bit) << (bit + 1)) | ((unsigned long long)val << bit) | lo;
}

// dst[e - off] = src[half_index(e)] (pack) or the reverse (unpack), e in [off, off + cnt),
// T = one 8- or 16-byte element; a grid-stride loop over a persistent grid.
template <typename T, bool PACK>
__global__ void __launch_bounds__(256) shard_copy(T *__restrict__ state, T *__restrict__ buf, uint32_t bit,
                                                  uint32_t val, unsigned long long off,
                                                  unsigned long long cnt) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += stride) {
        const unsigned long long i = half_index(e + off, bit, val);
        if (PACK)
            buf[e] = state[i];
        else
            state[i] = buf[e];
    }
}

}  // namespace svk

namespace {

sv_status shard_copy_launch(sv_state *s, uint32_t bit, uint32_t value, uint64_t offset, uint64_t count,
                            void *buf, bool pack, const char *who) {
    clear_error();
    if (!s || !buf) return set_error(SV_ERR_ARG, std::string(who) + ": null argument");
    if (check_live(s, who) != SV_OK) return SV_ERR_STATE;
    if (bit >= s->n || value > 1u) return set_error(SV_ERR_ARG, std::string(who) + ": bit must be < n, value 0 or 1");
    const uint64_t half = 1ull << (s->n - 1);
    if (offset > half || count > half - offset)
        return set_error(SV_ERR_ARG, std::string(who) + ": offset + count exceeds the half (2^(n-1) amplitudes)");
    if (count == 0) return SV_OK;
    const bool aligned16 = (reinterpret_cast<uintptr_t>(buf) & 15u) == 0;
    const unsigned grid = (unsigned)std::max(1, s->num_sms) * 8u;
    if (s->dtype == SV_C128) {
        if (!aligned16) return set_error(SV_ERR_ARG, std::string(who) + ": buffer must be 16-byte aligned");
        auto *st = static_cast<uint4 *>(s->buf);
        auto *b = static_cast<uint4 *>(buf);
        const unsigned g = (unsigned)std::min<uint64_t>(grid, (count + 255) / 256);
        if (pack) svk::shard_copy<uint4, true><<<g, 256, 0, s->stream>>>(st, b, bit, value, offset, count);
        else svk::shard_copy<uint4, false><<<g, 256, 0, s->stream>>>(st, b, bit, value, offset, count);
    } else if (bit >= 1 && aligned16 && (offset % 2 == 0) && (count % 2 == 0)) {
        // complex64 amplitudes in pairs: bit >= 1 keeps a pair together
        auto *st = static_cast<uint4 *>(s->buf);
        auto *b = static_cast<uint4 *>(buf);
        const unsigned g = (unsigned)std::min<uint64_t>(grid, (count / 2 + 255) / 256);
        if (pack) svk::shard_copy<uint4, true><<<g, 256, 0, s->stream>>>(st, b, bit - 1, value, offset / 2, count / 2);
        else svk::shard_copy<uint4, false><<<g, 256, 0, s->stream>>>(st, b, bit - 1, value, offset / 2, count / 2);
    } else {
        if (reinterpret_cast<uintptr_t>(buf) & 7u)
            return set_error(SV_ERR_ARG, std::string(who) + ": buffer must be 8-byte aligned");
        auto *st = static_cast<uint2 *>(s->buf);
        auto *b = static_cast<uint2 *>(buf);
        const unsigned g = (unsigned)std::min<uint64_t>(grid, (count + 255) / 256);
        if (pack) svk::shard_copy<uint2, true><<<g, 256, 0, s->stream>>>(st, b, bit, value, offset, count);
        else svk::shard_copy<uint2, false><<<g, 256, 0, s->stream>>>(st, b, bit, value, offset, count);
    }
    SV_CUDA(cudaGetLastError());
    if (!pack) s->basis_known = false;
    return SV_OK;
}

}  // namespace

extern "C" {

sv_status sv_shard_pack(sv_state *s, uint32_t bit, uint32_t value, uint64_t offset, uint64_t count,
                        void *dst_dev) {
    return shard_copy_launch(s, bit, value, offset, count, dst_dev, true, "sv_shard_pack");
}

sv_status sv_shard_unpack(sv_state *s, uint32_t bit, uint32_t value, uint64_t offset, uint64_t count,
                          const void *src_dev) {
    return shard_copy_launch(s, bit, value, offset, count, const_cast<void *>(src_dev), false,
                             "sv_shard_unpack");
}

}  // extern "C"
