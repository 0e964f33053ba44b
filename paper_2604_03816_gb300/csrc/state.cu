// C-ABI implementation: states, fusion entry points, the precision controller and the
// apply / reduction calls.  Argument checking happens here; the kernels live in
// apply_kernels.cu and reduce_kernels.cu.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "sv_internal.h"

namespace svi {

static thread_local std::string g_err;

sv_status set_error(sv_status st, const std::string &msg) {
    g_err = msg;
    return st;
}
void clear_error() { g_err.clear(); }

static size_t elem_bytes(sv_dtype d) { return d == SV_C64 ? 8 : 16; }
static size_t state_bytes(const sv_state *s) { return elem_bytes(s->dtype) << s->n; }

sv_status check_device_error(sv_state *s) {
    SV_CUDA(cudaStreamSynchronize(s->stream));
    int err = 0;
    SV_CUDA(cudaMemcpy(&err, s->ws + WS_ERR, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != 0) {
        SV_CUDA(cudaMemset(s->ws + WS_ERR, 0, sizeof(int)));
        return set_error(SV_ERR_TIMEOUT, "a bounded device-side wait gave up (error word " +
                                             std::to_string(err) + ")");
    }
    return SV_OK;
}

static sv_status validate_gate(const sv_gate *g, uint32_t n, const char *who) {
    if (!g || !g->u) return set_error(SV_ERR_ARG, std::string(who) + ": null gate or matrix");
    if (g->k < 1 || g->k > SV_MAX_K)
        return set_error(SV_ERR_ARG, std::string(who) + ": gate width must be 1..5");
    uint64_t seen = 0;
    for (uint32_t j = 0; j < g->k; ++j) {
        if (g->targets[j] >= n)
            return set_error(SV_ERR_ARG, std::string(who) + ": target " +
                                             std::to_string(g->targets[j]) + " >= n");
        if (seen & (1ull << g->targets[j]))
            return set_error(SV_ERR_ARG, std::string(who) + ": repeated target");
        seen |= 1ull << g->targets[j];
    }
    return SV_OK;
}

// Test hook: the next g_fail_allocs state-buffer allocations fail (sv_debug_fail_allocs).
static std::atomic<uint32_t> g_fail_allocs{0};

static cudaError_t alloc_state_buffer(void **p, size_t bytes) {
    uint32_t left = g_fail_allocs.load();
    while (left > 0 && !g_fail_allocs.compare_exchange_weak(left, left - 1)) {
    }
    if (left > 0) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

// Give a library-owned state a buffer of `need` bytes.  The new buffer is allocated
// before the old one is released, so a failure leaves the state as it was; only if that
// fails is the old buffer released first and the allocation tried again.  If the second
// try fails too, the state has no buffer (buf == nullptr): every call but sv_set_dtype,
// sv_info and sv_free then returns SV_ERR_STATE instead of launching on it.
static sv_status replace_buffer(sv_state *s, size_t need, const char *who) {
    void *nb = nullptr;
    SV_CUDA(cudaStreamSynchronize(s->stream));
    cudaError_t e = alloc_state_buffer(&nb, need);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (s->buf) cudaFree(s->buf);
        s->buf = nullptr;
        s->cap = 0;
        e = alloc_state_buffer(&nb, need);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return set_error(SV_ERR_OOM, std::string(who) + ": no device memory for a state buffer of " +
                                             std::to_string(need) + " bytes; the state has no buffer "
                                             "now (sv_set_dtype allocates one again)");
        }
    } else if (s->buf) {
        SV_CUDA(cudaFree(s->buf));
    }
    s->buf = nb;
    s->cap = need;
    return SV_OK;
}

const std::vector<Gate> &narrow_schedule(const sv_circuit *c) {
    bool wide = false;
    for (const Gate &g : c->gates) wide = wide || g.k == 5;
    if (!wide || c->in_gates.empty()) return c->gates;
    std::call_once(c->narrow_once, [&] {
        c->narrow = fuse_gates(c->in_gates, c->n, std::min(c->max_k, 4u), nullptr,
                               (c->flags & SV_FUSE_COMMUTE) != 0);
    });
    return c->narrow;
}

// SV_ERR_STATE for a state left without a buffer by a failed reallocation.
sv_status check_live(const sv_state *s, const char *who) {
    if (!s->buf)
        return set_error(SV_ERR_STATE, std::string(who) + ": the state has no buffer (a reallocation "
                                                          "failed); call sv_set_dtype or sv_free");
    return SV_OK;
}

static sv_status measure_norm(sv_state *s, double *out) {
    double *res = reinterpret_cast<double *>(s->ws + WS_RESULT) + 63;
    sv_status st = launch_norm(s, res);
    if (st != SV_OK) return st;
    SV_CUDA(cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    return check_device_error(s);
}

}  // namespace svi

using namespace svi;

extern "C" {

const char *sv_last_error(void) { return g_err.c_str(); }

sv_status sv_alloc(uint32_t n, sv_dtype dtype, void *dev_buf, size_t bytes, void *stream,
                   sv_state **out) {
    clear_error();
    if (!out) return set_error(SV_ERR_ARG, "sv_alloc: null out");
    *out = nullptr;
    if (n < 1 || n > SV_MAX_QUBITS) return set_error(SV_ERR_ARG, "sv_alloc: n must be 1..34");
    if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "sv_alloc: bad dtype");
    const size_t need = elem_bytes(dtype) << n;
    if (dev_buf) {
        if (bytes < need) return set_error(SV_ERR_ARG, "sv_alloc: buffer smaller than 2^n amplitudes");
        if (reinterpret_cast<uintptr_t>(dev_buf) & 15u)
            return set_error(SV_ERR_ARG, "sv_alloc: buffer must be 16-byte aligned");
    }
    sv_state *s = new (std::nothrow) sv_state();
    if (!s) return set_error(SV_ERR_OOM, "sv_alloc: host allocation failed");
    s->n = n;
    s->dtype = dtype;
    s->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        delete s;
        return set_error(SV_ERR_CUDA, std::string("sv_alloc: ") + cudaGetErrorString(e));
    }
    if (dev_buf) {
        s->buf = dev_buf;
        s->cap = bytes;
        s->owned = false;
    } else {
        e = alloc_state_buffer(&s->buf, need);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            delete s;
            return set_error(SV_ERR_OOM, std::string("sv_alloc: state: ") + cudaGetErrorString(e));
        }
        s->cap = need;
        s->owned = true;
    }
    e = cudaMalloc(reinterpret_cast<void **>(&s->ws), WS_BYTES);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ws, 0, WS_BYTES, s->stream);
    if (e != cudaSuccess) {
        if (s->owned) cudaFree(s->buf);
        if (s->ws) cudaFree(s->ws);
        delete s;
        return set_error(SV_ERR_OOM, std::string("sv_alloc: workspace: ") + cudaGetErrorString(e));
    }
    sv_status st = sv_set_basis(s, 0);
    if (st != SV_OK) {
        sv_free(s);
        return st;
    }
    *out = s;
    return SV_OK;
}

sv_status sv_free(sv_state *s) {
    clear_error();
    if (!s) return SV_OK;
    cudaStreamSynchronize(s->stream);
    if (s->owned && s->buf) cudaFree(s->buf);
    if (s->ws) cudaFree(s->ws);
    if (s->snap) cudaFree(s->snap);
    if (s->samp) cudaFree(s->samp);
    if (s->probs_buf) cudaFree(s->probs_buf);
    delete s;
    return SV_OK;
}

sv_status sv_info(const sv_state *s, uint32_t *n, sv_dtype *dtype, void **dev_ptr) {
    clear_error();
    if (!s) return set_error(SV_ERR_ARG, "sv_info: null state");
    if (n) *n = s->n;
    if (dtype) *dtype = s->dtype;
    if (dev_ptr) *dev_ptr = s->buf;
    return SV_OK;
}

sv_status sv_set_basis(sv_state *s, uint64_t x) {
    clear_error();
    if (!s) return set_error(SV_ERR_ARG, "sv_set_basis: null state");
    if (check_live(s, "sv_set_basis") != SV_OK) return SV_ERR_STATE;
    if (x >> s->n) return set_error(SV_ERR_ARG, "sv_set_basis: x >= 2^n");
    SV_CUDA(cudaMemsetAsync(s->buf, 0, state_bytes(s), s->stream));
    sv_status st = launch_set_one(s, x);
    if (st != SV_OK) return st;
    s->basis_known = true;
    s->basis_x = x;
    return SV_OK;
}

sv_status sv_set_zero(sv_state *s) {
    clear_error();
    if (!s) return set_error(SV_ERR_ARG, "sv_set_zero: null state");
    if (check_live(s, "sv_set_zero") != SV_OK) return SV_ERR_STATE;
    SV_CUDA(cudaMemsetAsync(s->buf, 0, state_bytes(s), s->stream));
    s->basis_known = false;
    return SV_OK;
}

sv_status sv_set_dtype(sv_state *s, sv_dtype dtype) {
    clear_error();
    if (!s) return set_error(SV_ERR_ARG, "sv_set_dtype: null state");
    if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "sv_set_dtype: bad dtype");
    const size_t need = elem_bytes(dtype) << s->n;
    if (s->cap < need || !s->buf) {
        if (!s->owned)
            return set_error(SV_ERR_STATE, "sv_set_dtype: caller buffer too small for this dtype");
        const sv_status st = replace_buffer(s, need, "sv_set_dtype");
        if (st != SV_OK) return st;
    }
    s->dtype = dtype;
    return sv_set_basis(s, 0);
}

sv_status sv_set_state(sv_state *s, const void *src, int src_on_device) {
    clear_error();
    if (!s || !src) return set_error(SV_ERR_ARG, "sv_set_state: null argument");
    if (check_live(s, "sv_set_state") != SV_OK) return SV_ERR_STATE;
    SV_CUDA(cudaMemcpyAsync(s->buf, src, state_bytes(s),
                            src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s->stream));
    s->basis_known = false;
    if (!src_on_device) SV_CUDA(cudaStreamSynchronize(s->stream));
    return SV_OK;
}

sv_status sv_get_state(sv_state *s, void *dst, int dst_on_device) {
    clear_error();
    if (!s || !dst) return set_error(SV_ERR_ARG, "sv_get_state: null argument");
    if (check_live(s, "sv_get_state") != SV_OK) return SV_ERR_STATE;
    SV_CUDA(cudaMemcpyAsync(dst, s->buf, state_bytes(s),
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s->stream));
    if (!dst_on_device) return check_device_error(s);
    return SV_OK;
}

// A circuit object holding Algorithm 2's schedule of `in` and what sv_fuse_like needs.
static sv_status make_circuit(const std::vector<Gate> &in, uint32_t n, uint32_t max_k, sv_circuit **out,
                              const char *who, uint32_t flags = 0) {
    sv_circuit *c = new (std::nothrow) sv_circuit();
    if (!c) return set_error(SV_ERR_OOM, std::string(who) + ": host allocation failed");
    c->n = n;
    try {
        c->max_k = max_k;
        c->flags = flags;
        c->in_k.reserve(in.size());
        c->in_t.reserve(in.size() * SV_MAX_K);
        for (const Gate &g : in) {
            c->in_k.push_back(g.k);
            for (uint32_t j = 0; j < SV_MAX_K; ++j) c->in_t.push_back(j < g.k ? g.t[j] : 0);
            if (flags & SV_FUSE_COMMUTE) c->in_diag.push_back(diagonal_mask(g));
        }
        c->gates = fuse_gates(in, n, max_k, &c->plan, (flags & SV_FUSE_COMMUTE) != 0);
        c->in_gates = in;
    } catch (const std::bad_alloc &) {
        delete c;
        return set_error(SV_ERR_OOM, std::string(who) + ": host allocation failed");
    }
    *out = c;
    return SV_OK;
}

sv_status sv_fuse(const sv_gate *gates, size_t ngates, uint32_t n, uint32_t max_k,
                  sv_circuit **out) {
    return sv_fuse_ex(gates, ngates, n, max_k, 0, out);
}

sv_status sv_fuse_ex(const sv_gate *gates, size_t ngates, uint32_t n, uint32_t max_k, uint32_t flags,
                     sv_circuit **out) {
    clear_error();
    if (!out) return set_error(SV_ERR_ARG, "sv_fuse: null out");
    *out = nullptr;
    if (n < 1 || n > SV_MAX_QUBITS) return set_error(SV_ERR_ARG, "sv_fuse: n must be 1..34");
    if (max_k > SV_MAX_K) return set_error(SV_ERR_ARG, "sv_fuse: max_k must be 0..5");
    if (flags & ~SV_FUSE_COMMUTE) return set_error(SV_ERR_ARG, "sv_fuse_ex: unknown flag");
    if (ngates && !gates) return set_error(SV_ERR_ARG, "sv_fuse: null gates");
    std::vector<Gate> in;
    in.reserve(ngates);
    for (size_t i = 0; i < ngates; ++i) {
        sv_status st = validate_gate(&gates[i], n, "sv_fuse");
        if (st != SV_OK) return set_error(st, sv_last_error() + (" (gate " + std::to_string(i) + ")"));
        in.push_back(sorted_gate(gates[i].k, gates[i].targets, gates[i].u));
    }
    return make_circuit(in, n, max_k, out, "sv_fuse", flags);
}

// Density matrices with single-qubit depolarizing noise (Section 9.5): rho on n qubits as
// the 2n-qubit vector v[r + 2^n c] = rho[r, c].  rho -> U rho U^dagger is U on the row bits
// T and conj(U) on the column bits T + n; the channel (1 - p) rho + (p/3)(X rho X + Y rho Y
// + Z rho Z) on qubit q is the 4 x 4 matrix (1 - p) I + (p/3) sum_P conj(P) (x) P on the
// bits (q, q + n) (local bit 0 = row bit q), applied to each target right after the gate.
sv_status sv_fuse_density(const sv_gate *gates, size_t ngates, uint32_t n, double p, uint32_t max_k,
                          sv_circuit **out) {
    clear_error();
    if (!out) return set_error(SV_ERR_ARG, "sv_fuse_density: null out");
    *out = nullptr;
    if (n < 1 || 2 * n > SV_MAX_QUBITS)
        return set_error(SV_ERR_ARG, "sv_fuse_density: n must be 1..17 (2n <= 34 vector qubits)");
    if (max_k > SV_MAX_K) return set_error(SV_ERR_ARG, "sv_fuse_density: max_k must be 0..5");
    if (!(p >= 0.0 && p <= 1.0)) return set_error(SV_ERR_ARG, "sv_fuse_density: p must be in [0, 1]");
    if (ngates && !gates) return set_error(SV_ERR_ARG, "sv_fuse_density: null gates");
    // the channel's superoperator on (row bit, column bit), index l = r + 2 c
    const cplx I(0.0, 1.0);
    const cplx P[3][2][2] = {{{0.0, 1.0}, {1.0, 0.0}}, {{0.0, -I}, {I, 0.0}}, {{1.0, 0.0}, {0.0, -1.0}}};
    std::vector<cplx> chan(16, cplx(0.0, 0.0));
    for (int l2 = 0; l2 < 4; ++l2)
        for (int l = 0; l < 4; ++l) {
            const int r2 = l2 & 1, c2 = l2 >> 1, r = l & 1, c = l >> 1;
            cplx v = l2 == l ? cplx(1.0 - p, 0.0) : cplx(0.0, 0.0);
            for (int q = 0; q < 3; ++q) v += (p / 3.0) * P[q][r2][r] * std::conj(P[q][c2][c]);
            chan[l2 * 4 + l] = v;
        }
    std::vector<Gate> in;
    in.reserve(ngates * 4);
    for (size_t i = 0; i < ngates; ++i) {
        sv_status st = validate_gate(&gates[i], n, "sv_fuse_density");
        if (st != SV_OK) return set_error(st, sv_last_error() + (" (gate " + std::to_string(i) + ")"));
        const Gate g = sorted_gate(gates[i].k, gates[i].targets, gates[i].u);
        Gate gc = g;
        for (uint32_t j = 0; j < g.k; ++j) gc.t[j] = g.t[j] + n;
        for (cplx &v : gc.u) v = std::conj(v);
        in.push_back(g);
        in.push_back(gc);
        if (p > 0.0)
            for (uint32_t j = 0; j < g.k; ++j) {
                Gate d;
                d.k = 2;
                d.t[0] = g.t[j];
                d.t[1] = g.t[j] + n;
                d.u = chan;
                in.push_back(d);
            }
    }
    return make_circuit(in, 2 * n, max_k, out, "sv_fuse_density");
}

sv_status sv_fuse_like(const sv_circuit *pattern, const sv_gate *gates, size_t ngates, sv_circuit **out) {
    clear_error();
    if (!pattern || !out || (ngates && !gates)) return set_error(SV_ERR_ARG, "sv_fuse_like: null argument");
    *out = nullptr;
    if (ngates != pattern->in_k.size())
        return set_error(SV_ERR_ARG, "sv_fuse_like: gate count differs from the pattern's");
    std::vector<Gate> in;
    in.reserve(ngates);
    for (size_t i = 0; i < ngates; ++i) {
        sv_status st = validate_gate(&gates[i], pattern->n, "sv_fuse_like");
        if (st != SV_OK) return st;
        in.push_back(sorted_gate(gates[i].k, gates[i].targets, gates[i].u));
        const Gate &g = in.back();
        bool same = g.k == pattern->in_k[i];
        for (uint32_t j = 0; same && j < g.k; ++j) same = g.t[j] == pattern->in_t[i * SV_MAX_K + j];
        if (!same)
            return set_error(SV_ERR_ARG, "sv_fuse_like: gate " + std::to_string(i) +
                                             " acts on other qubits than the pattern's");
        if ((pattern->flags & SV_FUSE_COMMUTE) && diagonal_mask(g) != pattern->in_diag[i])
            return set_error(SV_ERR_ARG, "sv_fuse_like: gate " + std::to_string(i) +
                                             " commutes differently from the pattern's (its "
                                             "diagonal qubits differ)");
    }
    sv_circuit *c = new (std::nothrow) sv_circuit();
    if (!c) return set_error(SV_ERR_OOM, "sv_fuse_like: host allocation failed");
    try {
        c->n = pattern->n;
        c->max_k = pattern->max_k;
        c->flags = pattern->flags;
        c->in_k = pattern->in_k;
        c->in_t = pattern->in_t;
        c->in_diag = pattern->in_diag;
        c->plan = pattern->plan;
        c->in_gates = in;
        c->gates = replay_fusion(std::move(in), pattern->plan);
    } catch (const std::bad_alloc &) {
        delete c;
        return set_error(SV_ERR_OOM, "sv_fuse_like: host allocation failed");
    }
    *out = c;
    return SV_OK;
}

sv_status sv_circuit_free(sv_circuit *c) {
    delete c;
    return SV_OK;
}

sv_status sv_circuit_size(const sv_circuit *c, size_t *nfused, uint32_t *n) {
    clear_error();
    if (!c) return set_error(SV_ERR_ARG, "sv_circuit_size: null circuit");
    if (nfused) *nfused = c->gates.size();
    if (n) *n = c->n;
    return SV_OK;
}

sv_status sv_circuit_gate(const sv_circuit *c, size_t i, uint32_t *k, uint32_t *targets, double *u) {
    clear_error();
    if (!c || i >= c->gates.size()) return set_error(SV_ERR_ARG, "sv_circuit_gate: bad index");
    const Gate &g = c->gates[i];
    if (k) *k = g.k;
    if (targets)
        for (uint32_t j = 0; j < g.k; ++j) targets[j] = g.t[j];
    if (u)
        for (size_t j = 0; j < g.u.size(); ++j) {
            u[2 * j] = g.u[j].real();
            u[2 * j + 1] = g.u[j].imag();
        }
    return SV_OK;
}

static void plan_passes(const sv_state *s, const std::vector<Gate> &gates, size_t begin, size_t end,
                        std::vector<int> *first, std::vector<int> *second);

sv_status sv_plan_passes(const sv_circuit *c, uint32_t policy, uint32_t *first, int32_t *second,
                         size_t cap, size_t *npasses) {
    clear_error();
    if (!c || !first || !second || !npasses) return set_error(SV_ERR_ARG, "sv_plan_passes: null argument");
    sv_state tmp;                   // host description only: no device memory is touched
    tmp.n = c->n;
    tmp.dtype = SV_C64;
    tmp.policy = policy;
    std::vector<int> f, sc;
    plan_passes(&tmp, c->gates, 0, c->gates.size(), &f, &sc);
    *npasses = f.size();
    if (cap < f.size()) return set_error(SV_ERR_ARG, "sv_plan_passes: cap below the pass count");
    for (size_t i = 0; i < f.size(); ++i) {
        first[i] = (uint32_t)f[i];
        second[i] = sc[i];
    }
    return SV_OK;
}

sv_status sv_choose_dtype(uint32_t n, uint64_t g, double eps_tol, sv_dtype *out, double *eps_round) {
    clear_error();
    if (!out) return set_error(SV_ERR_ARG, "sv_choose_dtype: null out");
    const double e = (double)g * std::ldexp(1.0, (int)n) * 1.19e-7;   // Eq. 12
    *out = e <= eps_tol ? SV_C64 : SV_C128;
    if (eps_round) *eps_round = e;
    return SV_OK;
}

sv_status sv_gate_structure(const sv_gate *g, uint32_t *kind, uint32_t *control_mask) {
    clear_error();
    sv_status st = validate_gate(g, SV_MAX_QUBITS, "sv_gate_structure");
    if (st != SV_OK) return st;
    const Gate sg = sorted_gate(g->k, g->targets, g->u);
    const Structure s = classify(sg);
    uint32_t mask = 0;
    for (uint32_t i = 0; i < s.nctrl; ++i)
        for (uint32_t j = 0; j < g->k; ++j)
            if (g->targets[j] == s.ctrl_q[i]) mask |= 1u << j;
    if (kind) *kind = s.kind;
    if (control_mask) *control_mask = mask;
    return SV_OK;
}

sv_status sv_apply_gate(sv_state *s, const sv_gate *g) {
    clear_error();
    if (!s) return set_error(SV_ERR_ARG, "sv_apply_gate: null state");
    if (check_live(s, "sv_apply_gate") != SV_OK) return SV_ERR_STATE;
    sv_status st = validate_gate(g, s->n, "sv_apply_gate");
    if (st != SV_OK) return st;
    s->basis_known = false;
    return launch_apply(s, sorted_gate(g->k, g->targets, g->u));
}

// With SV_POLICY_TWO_GATE_PASSES: would launch_apply run g as a dense pass (tensor cores,
// or the CUDA cores for k <= 3) on this complex64 state, so that it may share a pass with
// another dense gate?
static bool pair_candidate(const sv_state *s, const Gate &g) {
    if (s->dtype != SV_C64 || !(s->policy & SV_POLICY_TWO_GATE_PASSES) || (s->policy & SV_POLICY_NO_TENSOR_CORES))
        return false;
    if (!(s->policy & SV_POLICY_DENSE_ONLY) && struct_preferred(s, classify(g))) return false;
    return true;
}

// The passes of gates [begin, end): each gate in schedule order starts a pass unless an
// earlier pass took it; a dense complex64 gate takes as its partner the first later dense
// gate (within a window of 64) whose predecessors in the DAG of Eq. 8 (the last earlier
// gate on each of its qubits) have all been applied, and whose targets fit one tile with
// its own.  The partner then commutes with every gate it passes over (they share no
// qubit), so the product of the passes is the schedule's.  first[i]: the gate that
// pass i starts with; second[i]: its partner or -1.
static void plan_passes(const sv_state *s, const std::vector<Gate> &gates, size_t begin, size_t end,
                        std::vector<int> *first, std::vector<int> *second) {
    const size_t m = end - begin;
    std::vector<char> cand(m), done(m, 0);
    std::vector<int> preds;                    // up to SV_MAX_K per gate, -1 = none
    preds.assign(m * SV_MAX_K, -1);
    std::vector<int> last(64, -1);
    bool any = false;
    for (size_t i = 0; i < m; ++i) {
        const Gate &g = gates[begin + i];
        cand[i] = pair_candidate(s, g);
        any = any || cand[i];
        for (uint32_t j = 0; j < g.k; ++j) {
            preds[i * SV_MAX_K + j] = last[g.t[j]];
            last[g.t[j]] = (int)i;
        }
    }
    first->clear();
    second->clear();
    const size_t window = 64;
    for (size_t i = 0; i < m; ++i) {
        if (done[i]) continue;
        done[i] = 1;
        int partner = -1;
        if (any && cand[i]) {
            for (size_t v = i + 1; v < m && v <= i + window; ++v) {
                if (done[v] || !cand[v]) continue;
                bool ready = true;
                for (uint32_t j = 0; j < SV_MAX_K && ready; ++j) {
                    const int p = preds[v * SV_MAX_K + j];
                    ready = p < 0 || done[p];
                }
                if (!ready || !tc2_pair_fits(s, gates[begin + i], gates[begin + v])) continue;
                partner = (int)v;
                done[v] = 1;
                break;
            }
        }
        first->push_back((int)(begin + i));
        second->push_back(partner < 0 ? -1 : (int)(begin + partner));
    }
}

// Enqueue the passes of gates [begin, end).  With `timing`, CUDA events on the state's
// stream bracket the passes and their elapsed time is added to *ms (this synchronises on
// the events).
static sv_status run_schedule(sv_state *s, const std::vector<Gate> &gates, size_t begin, size_t end,
                              bool timing, sv_apply_report *r) {
    std::vector<int> first, second;
    plan_passes(s, gates, begin, end, &first, &second);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timing) {
        SV_CUDA(cudaEventCreate(&e0));
        SV_CUDA(cudaEventCreate(&e1));
        SV_CUDA(cudaEventRecord(e0, s->stream));
    }
    sv_status st = SV_OK;
    for (size_t i = 0; i < first.size() && st == SV_OK; ++i) {
        const Gate &g = gates[first[i]];
        if (second[i] >= 0) {
            const Gate &g2 = gates[second[i]];
            st = launch_apply_tc2(s, g, g2);
            r->bytes += 2ull * (8ull << s->n);
            ++r->tc_passes;
            ++r->paired_passes;
            r->max_k_used = std::max(r->max_k_used, std::max(g.k, g2.k));
            continue;
        }
        uint64_t b = 0;
        int kind = PASS_CUDA_CORE;
        st = launch_apply(s, g, &b, &kind);
        r->bytes += b;
        if (kind == PASS_TENSOR_CORE) ++r->tc_passes;
        r->max_k_used = std::max(r->max_k_used, g.k);
    }
    r->passes += first.size();
    if (timing) {
        cudaError_t e = cudaEventRecord(e1, s->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess && st == SV_OK)
            st = set_error(SV_ERR_CUDA, std::string("apply timing: ") + cudaGetErrorString(e));
        r->apply_ms += ms;
    }
    return st;
}

// The schedule a state of this dtype runs.  The complex128 tensor-core kernel takes gates
// of up to four qubits; width-5 gates would run on the FP64 CUDA cores at a small
// fraction of its rate, so complex128 states run the circuit's input gates fused again
// at width <= 4 (same flags; Algorithm 2 is deterministic, so this schedule is fixed by
// the circuit and built once).
static const std::vector<Gate> &schedule_for(const sv_state *s, const sv_circuit *c) {
    if (s->dtype != SV_C128 || (s->policy & SV_POLICY_NO_TENSOR_CORES) || !tc64_eligible(s, Gate()))
        return c->gates;
    return narrow_schedule(c);
}

sv_status sv_apply_circuit(sv_state *s, const sv_circuit *c, const sv_apply_opts *opts,
                           sv_apply_report *rep) {
    clear_error();
    if (!s || !c) return set_error(SV_ERR_ARG, "sv_apply_circuit: null argument");
    if (check_live(s, "sv_apply_circuit") != SV_OK) return SV_ERR_STATE;
    if (c->n != s->n) return set_error(SV_ERR_ARG, "sv_apply_circuit: circuit built for another n");
    for (const Gate &g : c->gates)
        if (g.k > s->n) return set_error(SV_ERR_ARG, "sv_apply_circuit: gate wider than the state");
    sv_apply_report r;
    std::memset(&r, 0, sizeof(r));
    r.dtype_used = s->dtype;
    const size_t G = c->gates.size();
    const bool adaptive = opts && opts->adaptive && s->dtype == SV_C64;
    const bool timing = opts && opts->timing;
    if (!adaptive) {
        s->basis_known = false;
        sv_status st = run_schedule(s, schedule_for(s, c), 0, schedule_for(s, c).size(), timing, &r);
        if (st != SV_OK) return st;
        if (rep) *rep = r;
        return SV_OK;
    }
    const double thr = opts->drift_threshold > 0 ? opts->drift_threshold : 1e-6;
    const size_t every = opts->drift_check_every;
    // Remember the initial state for a replay: a basis index or a snapshot.
    const bool from_basis = s->basis_known;
    const uint64_t x0 = s->basis_x;
    const size_t bytes64 = size_t(8) << s->n;
    if (!from_basis) {
        if (s->snap_cap < bytes64) {
            if (s->snap) cudaFree(s->snap);
            s->snap = nullptr;
            s->snap_cap = 0;
            SV_CUDA(cudaMalloc(&s->snap, bytes64));
            s->snap_cap = bytes64;
        }
        SV_CUDA(cudaMemcpyAsync(s->snap, s->buf, bytes64, cudaMemcpyDeviceToDevice, s->stream));
    }
    // a basis state |x> holds one amplitude 1 + 0i: its norm is exactly 1, no pass needed
    sv_status st = from_basis ? SV_OK : measure_norm(s, &r.norm_before);
    if (from_basis) r.norm_before = 1.0;
    if (st != SV_OK) return st;
    s->basis_known = false;
    bool promote = false;
    size_t done = 0;
    while (done < G && !promote) {
        const size_t next = every ? std::min(G, done + every) : G;
        st = run_schedule(s, c->gates, done, next, timing, &r);
        if (st != SV_OK) return st;
        done = next;
        st = measure_norm(s, &r.norm_after);
        if (st != SV_OK) return st;
        r.drift = std::fabs(r.norm_after - r.norm_before);
        promote = r.drift > thr;
    }
    if (promote) {
        // Replay the whole schedule in complex128 from the initial state.
        const size_t bytes128 = size_t(16) << s->n;
        if (s->cap < bytes128) {
            if (!s->owned)
                return set_error(SV_ERR_STATE, "sv_apply_circuit: promotion to complex128 needs a "
                                               "caller buffer of 2^n * 16 bytes");
            st = replace_buffer(s, bytes128, "sv_apply_circuit (promotion to complex128)");
            if (st != SV_OK) return st;
        }
        s->dtype = SV_C128;
        if (from_basis) {
            st = sv_set_basis(s, x0);
        } else {
            st = launch_widen(s, s->snap, s->buf);
        }
        if (st != SV_OK) return st;
        s->basis_known = false;
        r.max_k_used = 0;
        const std::vector<Gate> &replay = schedule_for(s, c);
        st = run_schedule(s, replay, 0, replay.size(), timing, &r);
        if (st != SV_OK) return st;
        r.promotions = 1;
        r.dtype_used = SV_C128;
        st = measure_norm(s, &r.norm_after);
        if (st != SV_OK) return st;
        r.drift = std::fabs(r.norm_after - r.norm_before);
    }
    if (rep) *rep = r;
    return SV_OK;
}

sv_status sv_norm(sv_state *s, double *out) {
    clear_error();
    if (!s || !out) return set_error(SV_ERR_ARG, "sv_norm: null argument");
    if (check_live(s, "sv_norm") != SV_OK) return SV_ERR_STATE;
    return measure_norm(s, out);
}

sv_status sv_probs(sv_state *s, void *out, int out_on_device) {
    clear_error();
    if (!s || !out) return set_error(SV_ERR_ARG, "sv_probs: null argument");
    if (check_live(s, "sv_probs") != SV_OK) return SV_ERR_STATE;
    if (out_on_device) return launch_probs(s, out);
    cudaPointerAttributes pa;
    const bool pinned = cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                        pa.devicePointer != nullptr;
    (void)cudaGetLastError();   // a pageable pointer is not an error
    const size_t pbytes = size_t(s->dtype == SV_C64 ? 4 : 8) << s->n;
    if (pinned && (s->policy & SV_POLICY_STAGED_PROBS)) {
        // through a device buffer kept by the state and one copy-engine transfer: the
        // kernel is a short HBM pass and the link transfer occupies no SM, so passes of
        // other streams run meanwhile
        if (s->probs_cap < pbytes) {
            if (s->probs_buf) cudaFree(s->probs_buf);
            s->probs_buf = nullptr;
            s->probs_cap = 0;
            SV_CUDA(cudaMalloc(&s->probs_buf, pbytes));
            s->probs_cap = pbytes;
        }
        sv_status st = launch_probs(s, s->probs_buf);
        if (st != SV_OK) return st;
        SV_CUDA(cudaMemcpyAsync(out, s->probs_buf, pbytes, cudaMemcpyDeviceToHost, s->stream));
        return check_device_error(s);
    }
    if (pinned) {
        // Pinned (page-locked, device-mapped) host memory: the kernel writes it directly
        // over the CPU-GPU link, with no device temporary and no separate copy.
        const sv_status st = launch_probs(s, pa.devicePointer);
        if (st != SV_OK) return st;
        return check_device_error(s);
    }
    const size_t bytes = pbytes;
    void *tmp = nullptr;
    SV_CUDA(cudaMallocAsync(&tmp, bytes, s->stream));
    sv_status st = launch_probs(s, tmp);
    if (st == SV_OK) {
        cudaError_t e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) st = set_error(SV_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFreeAsync(tmp, s->stream);
    if (st != SV_OK) return st;
    return check_device_error(s);
}

sv_status sv_density_probs(sv_state *s, void *out, int out_on_device) {
    clear_error();
    if (!s || !out) return set_error(SV_ERR_ARG, "sv_density_probs: null argument");
    if (check_live(s, "sv_density_probs") != SV_OK) return SV_ERR_STATE;
    if (s->n % 2) return set_error(SV_ERR_ARG, "sv_density_probs: the state is not a vectorised density matrix (odd width)");
    if (out_on_device) return launch_density_probs(s, out);
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr) {
        const sv_status st = launch_density_probs(s, pa.devicePointer);
        if (st != SV_OK) return st;
        return check_device_error(s);
    }
    (void)cudaGetLastError();
    const size_t bytes = size_t(s->dtype == SV_C64 ? 4 : 8) << (s->n / 2);
    void *tmp = nullptr;
    SV_CUDA(cudaMallocAsync(&tmp, bytes, s->stream));
    sv_status st = launch_density_probs(s, tmp);
    if (st == SV_OK) {
        cudaError_t e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) st = set_error(SV_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFreeAsync(tmp, s->stream);
    if (st != SV_OK) return st;
    return check_device_error(s);
}

sv_status sv_expect(sv_state *s, const uint64_t *xmask, const uint64_t *zmask, const double *coef,
                    size_t nterms, double *out) {
    clear_error();
    if (!s || !out || (nterms && (!xmask || !zmask || !coef)))
        return set_error(SV_ERR_ARG, "sv_expect: null argument");
    if (check_live(s, "sv_expect") != SV_OK) return SV_ERR_STATE;
    const uint64_t lim = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
    for (size_t t = 0; t < nterms; ++t)
        if ((xmask[t] & ~lim) || (zmask[t] & ~lim))
            return set_error(SV_ERR_ARG, "sv_expect: Pauli mask names a qubit >= n");
    if (nterms == 0) {
        *out = 0.0;
        return SV_OK;
    }
    sv_status st = launch_expect(s, xmask, zmask, coef, nterms, out);
    if (st != SV_OK) return st;
    return check_device_error(s);
}

sv_status sv_topk(sv_state *s, uint32_t k, uint64_t *idx, double *p) {
    clear_error();
    if (!s || !idx || !p) return set_error(SV_ERR_ARG, "sv_topk: null argument");
    if (check_live(s, "sv_topk") != SV_OK) return SV_ERR_STATE;
    if (k < 1 || k > 64) return set_error(SV_ERR_ARG, "sv_topk: k must be 1..64");
    sv_status st = launch_topk(s, k, idx, p);
    if (st != SV_OK) return st;
    return check_device_error(s);
}

sv_status sv_debug_fail_allocs(uint32_t count) {
    clear_error();
    g_fail_allocs.store(count);
    return SV_OK;
}

sv_status sv_set_policy(sv_state *s, uint32_t flags) {
    clear_error();
    if (!s) return set_error(SV_ERR_ARG, "sv_set_policy: null state");
    if (flags & ~(SV_POLICY_NO_TENSOR_CORES | SV_POLICY_DENSE_ONLY | SV_POLICY_STAGED_PROBS |
                  SV_POLICY_TWO_GATE_PASSES))
        return set_error(SV_ERR_ARG, "sv_set_policy: unknown flag");
    s->policy = flags;
    return SV_OK;
}

sv_status sv_sync(sv_state *s) {
    clear_error();
    if (!s) return set_error(SV_ERR_ARG, "sv_sync: null state");
    if (check_live(s, "sv_sync") != SV_OK) return SV_ERR_STATE;
    return check_device_error(s);
}

}  // extern "C"
