// Structure-aware passes: gates whose matrix has control qubits, or whose remainder V is
// diagonal or monomial (the exact structure of structure.cpp), applied without
// densifying them.  The paper fuses every gate into a dense unitary and leaves this
// structure and commutativity unused (Sections 10-11).
//
// With controls C and remainder V on targets T, U changes only the amplitudes whose C
// bits are all 1.  Every pass walks just that subspace: a work item's index gets 1 bits
// inserted at the control positions (and 0 bits at the positions of T for a per-group
// pass), so amplitudes with a control bit 0 are neither read nor written:
//
// * diagonal V: one thread per amplitude, psi[i] *= V[loc(i)][loc(i)]; entries exactly 1
//   are skipped (no load, no store), so e.g. a fused diagonal of phase gates that share
//   a qubit touches only the amplitudes it changes;
// * monomial V (row r has its one nonzero ph_r in column src_r): one thread per group,
//   out[r] = ph_r * in[src_r]; rows with src_r = r and ph_r = 1 are left alone, rows with
//   ph_r = 1 are plain moves;
// * dense V behind at least one control: one thread per group, out = V in, on the CUDA
//   cores (complex64 up to 4 targets; complex128 only when V has fewer targets than the
//   gate has controls, since GB300's FP64 pipe is narrow).
//
// These are streaming passes bound by HBM (complex128: by the FP64 pipe at about 4 FP64
// operations per amplitude, 74% of the copy bandwidth at best): a warp's loads cover
// contiguous runs of the state between the inserted bit positions.  c64 entries are the
// FP64 entries rounded to FP32; "exactly 1" is decided in the state's precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "sv_internal.h"

namespace svs {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }

// (a.x + i a.y)(b.x + i b.y): one product and one FMA per part.
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    return mk(fmar(a.x, b.x, -(a.y * b.y)), fmar(a.x, b.y, a.y * b.x));
}

// Bits inserted into a work item's index: positions p[0] < p[1] < ... (final positions
// in the state index), value 1 where bit i of `ones` is set.
struct Spread {
    uint32_t n = 0;
    uint32_t p[SV_MAX_K] = {0, 0, 0, 0, 0};
    uint32_t ones = 0;
};

__device__ __forceinline__ unsigned long long spread(unsigned long long x, const Spread &s) {
#pragma unroll
    for (int i = 0; i < SV_MAX_K; ++i)
        if (i < (int)s.n) {
            const uint32_t p = s.p[i];
            x = ((x >> p) << (p + 1)) | (x & ((1ull << p) - 1ull)) |
                ((unsigned long long)((s.ones >> i) & 1u) << p);
        }
    return x;
}

template <typename R>
struct DiagArgs {
    R d[2 << SV_MAX_K];          // V's diagonal (re, im)
    uint32_t one;                // bit r: entry r is exactly 1 in the state's precision
    void *psi;
    unsigned long long items;    // work items: VEC amplitudes each
    Spread sp;                   // the controls
    uint32_t k;                  // V's targets
    uint32_t t[SV_MAX_K];
};

template <typename R, int VEC> struct Vec;
template <> struct Vec<float, 1> { using T = float2; };
template <> struct Vec<float, 2> { using T = float4; };
template <> struct Vec<double, 1> { using T = double2; };
template <> struct Vec<double, 2> { using T = double4_16a; };

template <typename R>
__device__ __forceinline__ typename Cx<R>::T lane(const typename Vec<R, 1>::T &v, int) { return v; }
template <typename R>
__device__ __forceinline__ typename Cx<R>::T lane(const typename Vec<R, 2>::T &v, int q) {
    return q ? mk(v.z, v.w) : mk(v.x, v.y);
}
__device__ __forceinline__ void set_lane(float2 &v, int, float2 c) { v = c; }
__device__ __forceinline__ void set_lane(double2 &v, int, double2 c) { v = c; }
__device__ __forceinline__ void set_lane(float4 &v, int q, float2 c) {
    if (q) { v.z = c.x; v.w = c.y; } else { v.x = c.x; v.y = c.y; }
}
__device__ __forceinline__ void set_lane(double4_16a &v, int q, double2 c) {
    if (q) { v.z = c.x; v.w = c.y; } else { v.x = c.x; v.y = c.y; }
}

// A work item is VEC consecutive amplitudes (no control below bit log2(VEC)), moved with
// one vector access; it is skipped when all its entries are 1 and otherwise multiplied
// whole (a product with exactly 1 returns the amplitude, up to the sign of a zero).
template <typename R, int VEC>
__global__ void __launch_bounds__(256) apply_diag(const __grid_constant__ DiagArgs<R> a) {
    using C = typename Cx<R>::T;
    using V = typename Vec<R, VEC>::T;
    constexpr int ILP = 4;
    __shared__ C tab[1 << SV_MAX_K];
    if (threadIdx.x < (1u << a.k)) tab[threadIdx.x] = mk(a.d[2 * threadIdx.x], a.d[2 * threadIdx.x + 1]);
    __syncthreads();
    V *psi = reinterpret_cast<V *>(a.psi);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long e0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e0 < a.items;
         e0 += ILP * stride) {
        unsigned long long idx[ILP];
        uint32_t loc[ILP][VEC];
        V v[ILP];
        bool act[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const unsigned long long e = e0 + (unsigned long long)u * stride;
            const unsigned long long i0 = spread(e * VEC, a.sp);
            idx[u] = i0 / VEC;
            bool any = false;
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                uint32_t l = 0;
#pragma unroll
                for (int j = 0; j < SV_MAX_K; ++j)
                    if (j < (int)a.k) l |= (uint32_t)(((i0 + q) >> a.t[j]) & 1ull) << j;
                loc[u][q] = l;
                any |= !((a.one >> l) & 1u);
            }
            act[u] = e < a.items && any;
            if (act[u]) v[u] = psi[idx[u]];
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (!act[u]) continue;
            V w = v[u];
#pragma unroll
            for (int q = 0; q < VEC; ++q) set_lane(w, q, cmul(tab[loc[u][q]], lane<R>(v[u], q)));
            psi[idx[u]] = w;
        }
    }
}

template <typename R, int K>
struct MonoArgs {
    R ph[2 << K];                         // row r's entry (re, im)
    unsigned long long soff[1 << K];      // offset of row r's source member
    unsigned long long off[1 << K];       // offset of member r
    uint32_t skip, plain;                 // rows left alone / moved without a product
    void *psi;
    unsigned long long count;             // groups
    Spread sp;                            // V's targets (0) and the controls (1)
};

// Groups in flight per thread: several for narrow V (more loads in flight per thread).
template <typename R, int K>
__host__ __device__ constexpr int mono_ilp() { return K <= 2 ? 4 : (K == 3 ? 2 : 1); }

template <typename R, int K>
__global__ void __launch_bounds__(256) apply_mono(const __grid_constant__ MonoArgs<R, K> a) {
    using C = typename Cx<R>::T;
    constexpr int D = 1 << K, ILP = mono_ilp<R, K>();
    C *psi = reinterpret_cast<C *>(a.psi);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long g0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g0 < a.count;
         g0 += ILP * stride) {
        unsigned long long b[ILP];
        C v[ILP][D];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const unsigned long long g = g0 + (unsigned long long)u * stride;
            b[u] = spread(g, a.sp);
            if (g < a.count) {
#pragma unroll
                for (int r = 0; r < D; ++r)
                    if (!((a.skip >> r) & 1u)) v[u][r] = psi[b[u] + a.soff[r]];
            }
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (g0 + (unsigned long long)u * stride >= a.count) continue;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                if ((a.skip >> r) & 1u) continue;
                psi[b[u] + a.off[r]] =
                    ((a.plain >> r) & 1u) ? v[u][r] : cmul(mk(a.ph[2 * r], a.ph[2 * r + 1]), v[u][r]);
            }
        }
    }
}

template <typename R, int K>
struct CtrlArgs {
    R u[2 << (2 * K)];                    // V, row-major (re, im)
    unsigned long long off[1 << K];
    void *psi;
    unsigned long long count;             // groups
    Spread sp;
};

template <typename R, int K>
__global__ void __launch_bounds__(256) apply_ctrl(const __grid_constant__ CtrlArgs<R, K> a) {
    using C = typename Cx<R>::T;
    constexpr int D = 1 << K;
    C *psi = reinterpret_cast<C *>(a.psi);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < a.count;
         g += stride) {
        const unsigned long long b = spread(g, a.sp);
        C v[D];
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = psi[b + a.off[c]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const R ur = a.u[2 * (r * D + c)], ui = a.u[2 * (r * D + c) + 1];
                re = fmar(ur, v[c].x, re);
                re = fmar(-ui, v[c].y, re);
                im = fmar(ur, v[c].y, im);
                im = fmar(ui, v[c].x, im);
            }
            psi[b + a.off[r]] = mk(re, im);
        }
    }
}

// Resident-block grid over `work` items (cached per kernel in *per_sm).
template <typename F>
static unsigned grid_for(F kern, int *per_sm, const sv_state *s, unsigned long long work) {
    if (*per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, 0) != cudaSuccess || b < 1) b = 1;
        *per_sm = b;
    }
    const unsigned long long cap = (unsigned long long)(*per_sm) * (unsigned long long)s->num_sms;
    return (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>((work + 255) / 256, cap));
}

// The controls (value 1) and, if with_targets, V's targets (value 0), ascending.
static Spread make_spread(const svi::Structure &st, bool with_targets) {
    Spread sp;
    uint32_t pos[2 * SV_MAX_K], val[2 * SV_MAX_K], m = 0;
    for (uint32_t i = 0; i < st.nctrl; ++i) { pos[m] = st.ctrl_q[i]; val[m++] = 1; }
    if (with_targets)
        for (uint32_t j = 0; j < st.v.k; ++j) { pos[m] = st.v.t[j]; val[m++] = 0; }
    for (uint32_t i = 1; i < m; ++i)          // insertion sort by position
        for (uint32_t j = i; j > 0 && pos[j - 1] > pos[j]; --j) {
            std::swap(pos[j - 1], pos[j]);
            std::swap(val[j - 1], val[j]);
        }
    sp.n = m;
    for (uint32_t i = 0; i < m; ++i) {
        sp.p[i] = pos[i];
        if (val[i]) sp.ones |= 1u << i;
    }
    return sp;
}

template <typename R>
static bool is_one(const svi::cplx &z) {
    return static_cast<R>(z.real()) == R(1) && static_cast<R>(z.imag()) == R(0);
}

template <typename R, int VEC>
static sv_status launch_diag_v(sv_state *s, const DiagArgs<R> &a) {
    static int per_sm = 0;
    const unsigned grid = grid_for(apply_diag<R, VEC>, &per_sm, s, (a.items + 3) / 4);
    apply_diag<R, VEC><<<grid, 256, 0, s->stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

template <typename R>
static sv_status launch_diag(sv_state *s, const svi::Structure &st, uint64_t *bytes) {
    DiagArgs<R> a;
    const uint32_t dv = 1u << st.v.k;
    uint32_t changed = 0;
    a.one = 0;
    for (uint32_t r = 0; r < dv; ++r) {
        const svi::cplx z = st.v.u[(size_t)r * dv + r];
        a.d[2 * r] = static_cast<R>(z.real());
        a.d[2 * r + 1] = static_cast<R>(z.imag());
        if (is_one<R>(z)) a.one |= 1u << r;
        else ++changed;
    }
    const unsigned long long count = 1ull << (s->n - st.nctrl);   // controlled subspace
    a.psi = s->buf;
    a.sp = make_spread(st, false);
    a.k = st.v.k;
    for (uint32_t j = 0; j < SV_MAX_K; ++j) a.t[j] = j < st.v.k ? st.v.t[j] : 0u;
    if (bytes) *bytes = 2ull * sizeof(R) * 2ull * (count >> st.v.k) * changed;
    if (changed == 0) return SV_OK;
    // pairs of amplitudes unless a control sits at bit 0 (or the subspace is one amplitude)
    const bool pairs = count >= 2 && !(st.nctrl && st.ctrl_q[0] == 0);
    a.items = pairs ? count / 2 : count;
    return pairs ? launch_diag_v<R, 2>(s, a) : launch_diag_v<R, 1>(s, a);
}

template <typename R, int K>
static sv_status launch_mono(sv_state *s, const svi::Structure &st, uint64_t *bytes) {
    static int per_sm = 0;
    constexpr uint32_t D = 1u << K;
    MonoArgs<R, K> a;
    a.skip = a.plain = 0;
    for (uint32_t r = 0; r < D; ++r) {
        unsigned long long o = 0;
        for (uint32_t j = 0; j < (uint32_t)K; ++j)
            if ((r >> j) & 1u) o |= 1ull << st.v.t[j];
        a.off[r] = o;
    }
    uint32_t moved = 0;
    for (uint32_t r = 0; r < D; ++r) {
        uint32_t c = 0;
        while (st.v.u[(size_t)r * D + c] == svi::cplx(0.0, 0.0)) ++c;   // the row's nonzero
        const svi::cplx z = st.v.u[(size_t)r * D + c];
        a.ph[2 * r] = static_cast<R>(z.real());
        a.ph[2 * r + 1] = static_cast<R>(z.imag());
        a.soff[r] = a.off[c];
        if (is_one<R>(z)) {
            a.plain |= 1u << r;
            if (c == r) a.skip |= 1u << r;
        }
        moved += !((a.skip >> r) & 1u);
    }
    a.psi = s->buf;
    a.count = 1ull << (s->n - st.nctrl - K);
    a.sp = make_spread(st, true);
    if (bytes) *bytes = 2ull * sizeof(R) * 2ull * a.count * moved;
    if (moved == 0) return SV_OK;
    const unsigned grid = grid_for(apply_mono<R, K>, &per_sm, s, (a.count + mono_ilp<R, K>() - 1) / mono_ilp<R, K>());
    apply_mono<R, K><<<grid, 256, 0, s->stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

template <typename R, int K>
static sv_status launch_ctrl(sv_state *s, const svi::Structure &st, uint64_t *bytes) {
    static int per_sm = 0;
    constexpr uint32_t D = 1u << K;
    CtrlArgs<R, K> a;
    for (uint32_t i = 0; i < D * D; ++i) {
        a.u[2 * i] = static_cast<R>(st.v.u[i].real());
        a.u[2 * i + 1] = static_cast<R>(st.v.u[i].imag());
    }
    for (uint32_t r = 0; r < D; ++r) {
        unsigned long long o = 0;
        for (uint32_t j = 0; j < (uint32_t)K; ++j)
            if ((r >> j) & 1u) o |= 1ull << st.v.t[j];
        a.off[r] = o;
    }
    a.psi = s->buf;
    a.count = 1ull << (s->n - st.nctrl - K);
    a.sp = make_spread(st, true);
    if (bytes) *bytes = 2ull * sizeof(R) * 2ull * a.count * D;
    const unsigned grid = grid_for(apply_ctrl<R, K>, &per_sm, s, a.count);
    apply_ctrl<R, K><<<grid, 256, 0, s->stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

template <typename R>
static sv_status launch_struct_t(sv_state *s, const svi::Structure &st, uint64_t *bytes) {
    if (st.kind == SV_STRUCT_DIAGONAL) return launch_diag<R>(s, st, bytes);
    if (st.kind == SV_STRUCT_MONOMIAL) {
        switch (st.v.k) {
            case 1: return launch_mono<R, 1>(s, st, bytes);
            case 2: return launch_mono<R, 2>(s, st, bytes);
            case 3: return launch_mono<R, 3>(s, st, bytes);
            case 4: return launch_mono<R, 4>(s, st, bytes);
            case 5: return launch_mono<R, 5>(s, st, bytes);
            default: break;
        }
    } else if (st.kind == SV_STRUCT_DENSE) {
        switch (st.v.k) {
            case 1: return launch_ctrl<R, 1>(s, st, bytes);
            case 2: return launch_ctrl<R, 2>(s, st, bytes);
            default: break;
        }
        // complex128 takes a dense remainder only with fewer targets than controls (<= 2)
        if constexpr (sizeof(R) == 4) switch (st.v.k) {
            case 3: return launch_ctrl<R, 3>(s, st, bytes);
            case 4: return launch_ctrl<R, 4>(s, st, bytes);
            default: break;
        }
    }
    return svi::set_error(SV_ERR_ARG, "apply: no structured kernel for this gate");
}

}  // namespace svs

namespace svi {

bool struct_preferred(const sv_state *s, const Structure &st) {
    if (st.kind != SV_STRUCT_DENSE) return true;
    if (st.nctrl == 0) return false;
    return s->dtype == SV_C64 ? st.v.k <= 4 : st.v.k < st.nctrl;
}

sv_status launch_apply_struct(sv_state *s, const Structure &st, uint64_t *bytes) {
    if (st.kind == SV_STRUCT_IDENTITY) {
        if (bytes) *bytes = 0;
        return SV_OK;
    }
    return s->dtype == SV_C64 ? svs::launch_struct_t<float>(s, st, bytes)
                              : svs::launch_struct_t<double>(s, st, bytes);
}

}  // namespace svi
