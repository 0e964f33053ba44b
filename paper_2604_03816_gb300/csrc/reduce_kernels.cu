// Read-only reductions over the state: norm (Eq. 1), Z-basis probabilities, Pauli
// expectations and the top-k outcomes, plus the small initialisation kernels.
//
// Every reduction reads the state once with 16-byte vector loads from a fixed-size
// grid (so the partial-sum layout, and therefore the FP64 result, is the same on every
// run), folds per-thread values in FP64, reduces each block with warp shuffles and
// finishes with a single-block pass over the block partials in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "ptx.cuh"
#include "sv_internal.h"

namespace svk {

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[RED_THREADS / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < RED_THREADS / 32 ? ws[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// |alpha|^2 in the state's precision: fl(fl(x*x) + fl(y*y)) with round-to-nearest and
// no contraction, one fixed formula shared by probs, norm and top-k (so that a host
// computing the same IEEE operations takes the same top-k decisions).
__device__ __forceinline__ float prob_of(float x, float y) {
    return __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
}
__device__ __forceinline__ double prob_of(double x, double y) {
    return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
}

// ---------------------------------------------------------------- norm

__global__ void norm_c64(const float4 *__restrict__ v, unsigned long long nvec, double *partial) {
    double acc = 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < nvec; i += 4 * stride) {
        float4 a = v[i], b = v[i + stride], c = v[i + 2 * stride], d = v[i + 3 * stride];
        const float sa = __fadd_rn(prob_of(a.x, a.y), prob_of(a.z, a.w));
        const float sb = __fadd_rn(prob_of(b.x, b.y), prob_of(b.z, b.w));
        const float sc = __fadd_rn(prob_of(c.x, c.y), prob_of(c.z, c.w));
        const float sd = __fadd_rn(prob_of(d.x, d.y), prob_of(d.z, d.w));
        // eight amplitudes summed pairwise in FP32, one FP64 operation per eight (the FP64
        // pipe of this GPU runs at about 1/64 of the FP32 rate)
        acc += (double)__fadd_rn(__fadd_rn(sa, sb), __fadd_rn(sc, sd));
    }
    for (; i < nvec; i += stride) {
        float4 a = v[i];
        acc += (double)__fadd_rn(prob_of(a.x, a.y), prob_of(a.z, a.w));
    }
    const double r = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void norm_c128(const double2 *__restrict__ v, unsigned long long n, double *partial) {
    double acc = 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        double2 a = v[i], b = v[i + stride], c = v[i + 2 * stride], d = v[i + 3 * stride];
        acc += prob_of(a.x, a.y) + prob_of(b.x, b.y) + prob_of(c.x, c.y) + prob_of(d.x, d.y);
    }
    for (; i < n; i += stride) acc += prob_of(v[i].x, v[i].y);
    const double r = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

// out[0] = sum of partial[0..n) in a fixed order (one block).
__global__ void sum_partials(const double *partial, int n, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    const double r = block_sum(acc);
    if (threadIdx.x == 0) out[0] = r;
}

// ---------------------------------------------------------------- probabilities

__global__ void probs_c64(const float4 *__restrict__ v, unsigned long long nvec, float2 *out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvec;
         i += stride) {
        const float4 a = v[i];
        out[i] = make_float2(prob_of(a.x, a.y), prob_of(a.z, a.w));
    }
}

__global__ void probs_c128(const double2 *__restrict__ v, unsigned long long n, double *out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride)
        out[i] = prob_of(v[i].x, v[i].y);
}

// Diagonal of a density matrix held as the 2m-qubit vector v[r + 2^m c] = rho[r, c]:
// p(x) = Re rho[x, x] = Re v[x (2^m + 1)], in the state's precision.
template <typename C, typename R>
__global__ void density_diag(const C *__restrict__ v, uint32_t m, R *__restrict__ out) {
    const unsigned long long M = 1ull << m;
    for (unsigned long long x = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; x < M;
         x += (unsigned long long)gridDim.x * blockDim.x)
        out[x] = v[x * (M + 1)].x;
}

// ---------------------------------------------------------------- Pauli expectation

constexpr int EXP_MAX_TERMS = 32;

// Terms sharing one X-part x.  cc = coef * i^{|x & z|} (complex, FP64).
struct ExpectArgs {
    unsigned long long x;
    unsigned long long z[EXP_MAX_TERMS];
    double ccr[EXP_MAX_TERMS], cci[EXP_MAX_TERMS];
    int nterms;
    int hb;                   // highest set bit of x (x != 0)
    unsigned long long npairs;
};

// sum_k Re[ conj(psi[k ^ x]) psi[k] w(k) ],  w(k) = sum_t cc_t (-1)^{|k & z_t|}.
// x = 0: sum_k |psi_k|^2 Re w(k).  x != 0: the pair (k, k ^ x) with bit hb of k clear
// contributes both of its orderings.
template <typename R>
__global__ void expect_kernel(const __grid_constant__ ExpectArgs a, const void *psi_, double *partial) {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C *psi = reinterpret_cast<const C *>(psi_);
    double acc = 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         i < a.npairs; i += stride) {
        if (a.x == 0) {
            const C v = psi[i];
            double w = 0.0;
            for (int t = 0; t < a.nterms; ++t)
                w += (__popcll(i & a.z[t]) & 1) ? -a.ccr[t] : a.ccr[t];
            acc += w * (double)prob_of(v.x, v.y);
        } else {
            const unsigned long long k = insert_zero64(i, (uint32_t)a.hb), k2 = k ^ a.x;
            const C p = psi[k], q = psi[k2];
            // conj(q) p and conj(p) q = conj(conj(q) p)
            const double re = (double)q.x * p.x + (double)q.y * p.y;
            const double im = (double)q.x * p.y - (double)q.y * p.x;
            double w1r = 0, w1i = 0, w2r = 0, w2i = 0;
            for (int t = 0; t < a.nterms; ++t) {
                const bool s1 = __popcll(k & a.z[t]) & 1, s2 = __popcll(k2 & a.z[t]) & 1;
                w1r += s1 ? -a.ccr[t] : a.ccr[t];
                w1i += s1 ? -a.cci[t] : a.cci[t];
                w2r += s2 ? -a.ccr[t] : a.ccr[t];
                w2i += s2 ? -a.cci[t] : a.cci[t];
            }
            // Re[(re + i im) w1] + Re[(re - i im) w2]
            acc += re * w1r - im * w1i + re * w2r + im * w2i;
        }
    }
    const double r = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

// complex64, up to NT terms of one X-part: per term FP32 partial sums over runs of eight
// elements (pairs when x != 0), one FP64 step per run and term.  With s_t(k) = (-1)^{|k &
// z_t|} and cc_t = ccr_t + i cci_t, a term contributes ccr_t sum_k s_t(k) |psi_k|^2 when
// x = 0, and for x != 0, per pair (k, k2 = k ^ x) with bit hb of k clear and
// c = conj(psi_k2) psi_k = re + i im:  ccr_t (s_t(k) + s_t(k2)) re - cci_t (s_t(k) - s_t(k2)) im.
template <int NT, bool PAIRS>
__global__ void expect_c64(const __grid_constant__ ExpectArgs a, const float2 *__restrict__ psi,
                           double *partial) {
    double A[NT], B[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) A[t] = B[t] = 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         i0 < a.npairs; i0 += 8 * stride) {
        float sa[NT], sb[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) sa[t] = sb[t] = 0.f;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const unsigned long long i = i0 + r * stride;
            if (i >= a.npairs) break;
            if constexpr (!PAIRS) {
                const float2 v = psi[i];
                const float pr = prob_of(v.x, v.y);
#pragma unroll
                for (int t = 0; t < NT; ++t)
                    sa[t] = __fadd_rn(sa[t], (__popcll(i & a.z[t]) & 1) ? -pr : pr);
            } else {
                const unsigned long long k = insert_zero64(i, (uint32_t)a.hb), k2 = k ^ a.x;
                const float2 p = psi[k], q = psi[k2];
                const float re = __fadd_rn(__fmul_rn(q.x, p.x), __fmul_rn(q.y, p.y));
                const float im = __fsub_rn(__fmul_rn(q.x, p.y), __fmul_rn(q.y, p.x));
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const bool s1 = __popcll(k & a.z[t]) & 1, s2 = __popcll(k2 & a.z[t]) & 1;
                    if (s1 == s2) sa[t] = __fadd_rn(sa[t], s1 ? -2.f * re : 2.f * re);
                    else sb[t] = __fadd_rn(sb[t], s1 ? -2.f * im : 2.f * im);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            A[t] += (double)sa[t];
            B[t] += (double)sb[t];
        }
    }
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < NT; ++t) acc += a.ccr[t] * A[t] - a.cci[t] * B[t];
    const double r = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

// ---------------------------------------------------------------- top-k

// (p, idx) order: larger p first, then smaller index.
template <typename P>
__device__ __forceinline__ bool better(P pa, unsigned long long ia, P pb, unsigned long long ib) {
    return pa > pb || (pa == pb && ia < ib);
}

// Keys of the top-k lists.  complex64 probabilities are FP32 values, compared in FP32 (the
// same decisions as on their exact FP64 widenings).  FP64 probabilities are compared as
// their IEEE bit patterns, which order non-negative doubles like their values, in 64-bit
// integer arithmetic: a warp-wide FP64 compare costs tens of cycles on this GPU.
template <typename P> __device__ __forceinline__ P empty_key();
template <> __device__ __forceinline__ float empty_key<float>() { return -1.f; }
template <> __device__ __forceinline__ unsigned long long empty_key<unsigned long long>() { return 0ull; }

__device__ __forceinline__ unsigned long long key_of(double p) {   // p >= 0
    return (unsigned long long)__double_as_longlong(p);
}
__device__ __forceinline__ double value_of(unsigned long long k) { return __longlong_as_double((long long)k); }
__device__ __forceinline__ double value_of(float k) { return (double)k; }

// One warp's 64 entries, two per lane, plus the current worst.  Empty entries hold
// (empty_key, ~0): they lose to every real entry.
template <typename P>
struct TopList {
    P p0, p1;
    unsigned long long i0, i1;
    P wp;
    unsigned long long wi;
    int wl, ws;    // lane and slot of the worst entry

    __device__ void init() {
        p0 = p1 = empty_key<P>();
        i0 = i1 = ~0ull;
        find_worst();
    }
    __device__ void find_worst() {
        const int lane = threadIdx.x & 31;
        // this lane's worse entry
        bool second = better(p0, i0, p1, i1);
        P p = second ? p1 : p0;
        unsigned long long ix = second ? i1 : i0;
        int l = lane, s = second ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const P op = __shfl_xor_sync(0xffffffffu, p, o);
            const unsigned long long oi = __shfl_xor_sync(0xffffffffu, ix, o);
            const int ol = __shfl_xor_sync(0xffffffffu, l, o);
            const int os = __shfl_xor_sync(0xffffffffu, s, o);
            if (better(p, ix, op, oi) || (p == op && ix == oi && (ol < l || (ol == l && os < s)))) {
                p = op; ix = oi; l = ol; s = os;
            }
        }
        wp = p; wi = ix; wl = l; ws = s;
    }
    // Offer one candidate per lane; all lanes of the warp must call.
    __device__ void offer(P p, unsigned long long ix, bool valid) {
        const int lane = threadIdx.x & 31;
        unsigned mask = __ballot_sync(0xffffffffu, valid && better(p, ix, wp, wi));
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const P cp = __shfl_sync(0xffffffffu, p, src);
            const unsigned long long ci = __shfl_sync(0xffffffffu, ix, src);
            if (!better(cp, ci, wp, wi)) continue;     // uniform across the warp
            if (lane == wl) {
                if (ws == 0) { p0 = cp; i0 = ci; } else { p1 = cp; i1 = ci; }
            }
            find_worst();
        }
    }
};

// Pass 1: each warp scans a contiguous chunk (a multiple of 256 amplitudes), eight
// amplitudes per lane per step from independent 16-byte loads; a step is offered to the
// warp's list only if some lane holds a probability not below the list's current worst.
// The block's warps then merge their lists, and the block writes 64 candidates.
template <typename R>
__global__ void __launch_bounds__(256) topk_pass1(const void *psi_, unsigned long long N,
                                                  unsigned long long chunk, double *cand_p,
                                                  unsigned long long *cand_i) {
    using Key = typename std::conditional<sizeof(R) == 4, float, unsigned long long>::type;
    __shared__ Key lp[8][64];
    __shared__ unsigned long long li[8][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    TopList<Key> L;
    L.init();
    const unsigned long long lo = warp * chunk, hi = min(N, lo + chunk);
    for (unsigned long long b = lo; b < hi; b += 256) {
        Key p[8];
        unsigned long long k[8];
        bool ok[8];
        if constexpr (sizeof(R) == 4) {
            // four float4 loads: amplitudes b + 2 (lane + 32 j) + {0, 1}
            const float4 *v4 = reinterpret_cast<const float4 *>(psi_);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const unsigned long long k0 = b + 2ull * (lane + 32 * j);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k0 < hi) v = v4[k0 >> 1];
                k[2 * j] = k0;
                k[2 * j + 1] = k0 + 1;
                ok[2 * j] = k0 < hi;
                ok[2 * j + 1] = k0 + 1 < hi;
                p[2 * j] = ok[2 * j] ? prob_of(v.x, v.y) : empty_key<Key>();
                p[2 * j + 1] = ok[2 * j + 1] ? prob_of(v.z, v.w) : empty_key<Key>();
            }
        } else {
            const double2 *v2 = reinterpret_cast<const double2 *>(psi_);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const unsigned long long k0 = b + lane + 32ull * j;
                double2 v = make_double2(0.0, 0.0);
                if (k0 < hi) v = v2[k0];
                k[j] = k0;
                ok[j] = k0 < hi;
                p[j] = ok[j] ? key_of(prob_of(v.x, v.y)) : empty_key<Key>();
            }
        }
        Key mx = p[0];
#pragma unroll
        for (int j = 1; j < 8; ++j) mx = mx > p[j] ? mx : p[j];
        if (!__any_sync(0xffffffffu, mx >= L.wp)) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) L.offer(p[j], k[j], ok[j]);
    }
    // merge the block's eight lists in warp 0
    lp[w][2 * lane] = L.p0; li[w][2 * lane] = L.i0;
    lp[w][2 * lane + 1] = L.p1; li[w][2 * lane + 1] = L.i1;
    __syncthreads();
    if (w == 0) {
        for (int o = 1; o < 8; ++o)
            for (int h = 0; h < 2; ++h) {
                const unsigned long long ci = li[o][32 * h + lane];
                L.offer(lp[o][32 * h + lane], ci, ci != ~0ull);
            }
        // candidates as doubles; empty entries as -1
        const unsigned long long base = (unsigned long long)blockIdx.x * 64;
        cand_p[base + 2 * lane] = L.i0 == ~0ull ? -1.0 : value_of(L.p0);
        cand_i[base + 2 * lane] = L.i0;
        cand_p[base + 2 * lane + 1] = L.i1 == ~0ull ? -1.0 : value_of(L.p1);
        cand_i[base + 2 * lane + 1] = L.i1;
    }
}

// Pass 2 (one block of 32 warps): each warp merges a strided share of the m candidates,
// warp 0 merges the 32 lists and writes the best 64, sorted.
__global__ void __launch_bounds__(1024) topk_pass2(const double *cand_p, const unsigned long long *cand_i,
                                                   unsigned long long m, double *out_p,
                                                   unsigned long long *out_i) {
    __shared__ unsigned long long sp[32][64];
    __shared__ unsigned long long si[32][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TopList<unsigned long long> L;
    L.init();
    for (unsigned long long b = (unsigned long long)w * 32; b < m; b += 32ull * 32) {
        const unsigned long long j = b + lane;
        const bool ok = j < m;
        const unsigned long long kb = ok ? (unsigned long long)__double_as_longlong(cand_p[j]) : 0ull;
        const bool real = ok && !(kb >> 63);              // empty entries are -1
        L.offer(real ? kb : 0ull, real ? cand_i[j] : ~0ull, real);
    }
    sp[w][2 * lane] = L.p0; si[w][2 * lane] = L.i0;
    sp[w][2 * lane + 1] = L.p1; si[w][2 * lane + 1] = L.i1;
    __syncthreads();
    if (w != 0) return;
    for (int o = 1; o < 32; ++o)
        for (int h = 0; h < 2; ++h) {
            const unsigned long long ci = si[o][32 * h + lane];
            L.offer(sp[o][32 * h + lane], ci, ci != ~0ull);
        }
    sp[0][2 * lane] = L.p0; si[0][2 * lane] = L.i0;
    sp[0][2 * lane + 1] = L.p1; si[0][2 * lane + 1] = L.i1;
    __syncwarp();
    if (lane == 0) {
        unsigned long long *qp = sp[0];
        unsigned long long *qi = si[0];
        for (int a = 1; a < 64; ++a) {          // insertion sort, best first
            const unsigned long long p = qp[a];
            const unsigned long long ix = qi[a];
            int b = a - 1;
            while (b >= 0 && better(p, ix, qp[b], qi[b])) {
                qp[b + 1] = qp[b]; qi[b + 1] = qi[b];
                --b;
            }
            qp[b + 1] = p; qi[b + 1] = ix;
        }
        for (int a = 0; a < 64; ++a) {
            out_p[a] = qi[a] == ~0ull ? -1.0 : value_of(qp[a]);
            out_i[a] = qi[a];
        }
    }
}

// ---------------------------------------------------------------- init helpers

__global__ void set_amp_one(void *psi, unsigned long long x, int is_c128) {
    if (is_c128) reinterpret_cast<double2 *>(psi)[x] = make_double2(1.0, 0.0);
    else reinterpret_cast<float2 *>(psi)[x] = make_float2(1.0f, 0.0f);
}

__global__ void widen_kernel(const float2 *__restrict__ src, double2 *__restrict__ dst,
                             unsigned long long n) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride)
        dst[i] = make_double2((double)src[i].x, (double)src[i].y);
}

}  // namespace svk

namespace svi {

static int red_blocks(const sv_state *s) { return std::min(WS_NPARTIAL, s->num_sms * 8); }

sv_status launch_norm(sv_state *s, double *dev_out) {
    double *partial = reinterpret_cast<double *>(s->ws + WS_PARTIAL);
    const unsigned long long N = 1ull << s->n;
    const int nb = red_blocks(s);
    if (s->dtype == SV_C64)
        svk::norm_c64<<<nb, svk::RED_THREADS, 0, s->stream>>>(
            reinterpret_cast<const float4 *>(s->buf), N / 2, partial);
    else
        svk::norm_c128<<<nb, svk::RED_THREADS, 0, s->stream>>>(
            reinterpret_cast<const double2 *>(s->buf), N, partial);
    SV_CUDA(cudaGetLastError());
    svk::sum_partials<<<1, svk::RED_THREADS, 0, s->stream>>>(partial, nb, dev_out);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

sv_status launch_probs(sv_state *s, void *dev_out) {
    const unsigned long long N = 1ull << s->n;
    const int nb = s->num_sms * 8;
    if (s->dtype == SV_C64)
        svk::probs_c64<<<nb, 256, 0, s->stream>>>(reinterpret_cast<const float4 *>(s->buf), N / 2,
                                                   reinterpret_cast<float2 *>(dev_out));
    else
        svk::probs_c128<<<nb, 256, 0, s->stream>>>(reinterpret_cast<const double2 *>(s->buf), N,
                                                    reinterpret_cast<double *>(dev_out));
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

sv_status launch_density_probs(sv_state *s, void *dev_out) {
    const uint32_t m = s->n / 2;
    const int nb = s->num_sms * 8;
    if (s->dtype == SV_C64)
        svk::density_diag<<<nb, 256, 0, s->stream>>>(reinterpret_cast<const float2 *>(s->buf), m,
                                                     reinterpret_cast<float *>(dev_out));
    else
        svk::density_diag<<<nb, 256, 0, s->stream>>>(reinterpret_cast<const double2 *>(s->buf), m,
                                                     reinterpret_cast<double *>(dev_out));
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

sv_status launch_expect(sv_state *s, const uint64_t *x, const uint64_t *z, const double *c,
                        size_t nterms, double *host_out) {
    // group terms by X-part; each launch handles up to EXP_MAX_TERMS terms of one group
    std::vector<size_t> order(nterms);
    for (size_t i = 0; i < nterms; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return x[a] < x[b]; });
    double *partial = reinterpret_cast<double *>(s->ws + WS_PARTIAL);
    double *results = reinterpret_cast<double *>(s->ws + WS_RESULT);
    const int nb = red_blocks(s);
    double total = 0.0;
    size_t i = 0;
    while (i < nterms) {
        int nres = 0;
        while (i < nterms && nres < 64) {
            svk::ExpectArgs a;
            std::memset(&a, 0, sizeof(a));
            a.x = x[order[i]];
            a.nterms = 0;
            while (i < nterms && x[order[i]] == a.x && a.nterms < svk::EXP_MAX_TERMS) {
                const size_t t = order[i++];
                const int y = __builtin_popcountll(a.x & z[t]) & 3;   // i^y
                const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
                a.z[a.nterms] = z[t];
                a.ccr[a.nterms] = c[t] * re[y];
                a.cci[a.nterms] = c[t] * im[y];
                ++a.nterms;
            }
            if (a.x == 0) {
                a.hb = 0;
                a.npairs = 1ull << s->n;
            } else {
                a.hb = 63 - __builtin_clzll(a.x);
                a.npairs = 1ull << (s->n - 1);
            }
            if (s->dtype == SV_C64) {
                const float2 *v = reinterpret_cast<const float2 *>(s->buf);
                const bool pr = a.x != 0;
                switch (a.nterms) {
                    case 1: pr ? svk::expect_c64<1, true><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial)
                               : svk::expect_c64<1, false><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial); break;
                    case 2: pr ? svk::expect_c64<2, true><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial)
                               : svk::expect_c64<2, false><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial); break;
                    case 3: pr ? svk::expect_c64<3, true><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial)
                               : svk::expect_c64<3, false><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial); break;
                    case 4: pr ? svk::expect_c64<4, true><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial)
                               : svk::expect_c64<4, false><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, v, partial); break;
                    default: svk::expect_kernel<float><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, s->buf, partial);
                }
            } else
                svk::expect_kernel<double><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, s->buf, partial);
            SV_CUDA(cudaGetLastError());
            svk::sum_partials<<<1, svk::RED_THREADS, 0, s->stream>>>(partial, nb, results + nres);
            SV_CUDA(cudaGetLastError());
            ++nres;
        }
        double h[64];
        SV_CUDA(cudaMemcpyAsync(h, results, sizeof(double) * nres, cudaMemcpyDeviceToHost, s->stream));
        SV_CUDA(cudaStreamSynchronize(s->stream));
        for (int r = 0; r < nres; ++r) total += h[r];
    }
    *host_out = total;
    return SV_OK;
}

// Enqueue the top-64 search and asynchronous copies of the 64 (p, index) pairs, best
// first, into host_p / host_i (pinned memory for a truly asynchronous copy).
sv_status enqueue_topk(sv_state *s, double *host_p, unsigned long long *host_i) {
    const unsigned long long N = 1ull << s->n;
    const int threads = 256, warps_per_block = threads / 32;
    int blocks = std::min(s->num_sms * 4, TOPK_MAX_WARPS / warps_per_block);
    unsigned long long nwarps = (unsigned long long)blocks * warps_per_block;
    unsigned long long chunk = (N + nwarps - 1) / nwarps;
    chunk = (chunk + 255) / 256 * 256;
    double *cp = reinterpret_cast<double *>(s->ws + WS_TOPK);
    unsigned long long *ci = reinterpret_cast<unsigned long long *>(s->ws + WS_TOPK) + TOPK_MAX_WARPS * 64;
    double *op = reinterpret_cast<double *>(s->ws + WS_TOPK + WS_TOPK_BYTES);
    unsigned long long *oi = reinterpret_cast<unsigned long long *>(op + 64);
    if (s->dtype == SV_C64)
        svk::topk_pass1<float><<<blocks, threads, 0, s->stream>>>(s->buf, N, chunk, cp, ci);
    else
        svk::topk_pass1<double><<<blocks, threads, 0, s->stream>>>(s->buf, N, chunk, cp, ci);
    SV_CUDA(cudaGetLastError());
    svk::topk_pass2<<<1, 1024, 0, s->stream>>>(cp, ci, (unsigned long long)blocks * 64, op, oi);
    SV_CUDA(cudaGetLastError());
    SV_CUDA(cudaMemcpyAsync(host_p, op, 64 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SV_CUDA(cudaMemcpyAsync(host_i, oi, 64 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            s->stream));
    return SV_OK;
}

sv_status launch_topk(sv_state *s, uint32_t k, uint64_t *idx, double *p) {
    const unsigned long long N = 1ull << s->n;
    double hp[64];
    unsigned long long hi[64];
    sv_status st = enqueue_topk(s, hp, hi);
    if (st != SV_OK) return st;
    SV_CUDA(cudaStreamSynchronize(s->stream));
    const uint32_t m = (uint32_t)std::min<unsigned long long>(k, N);
    for (uint32_t j = 0; j < m; ++j) {
        idx[j] = hi[j];
        p[j] = hp[j];
    }
    return SV_OK;
}

// Enqueue sum_t coef[t] <P_t> for a raw device state into *out_dev, with block partials
// in caller-provided scratch (nb_fixed doubles per batch of up to EXP_MAX_TERMS terms
// sharing one X-part).  Uses no heap memory: the term order lives on the stack, so
// nterms is limited to ENQ_MAX_TERMS.  SV_ERR_ARG if the batches need more scratch.
sv_status enqueue_expect_sum(const void *psi, uint32_t n, sv_dtype dtype, const uint64_t *x,
                             const uint64_t *z, const double *c, size_t nterms, double *scratch,
                             size_t scratch_doubles, int nb_fixed, double *out_dev,
                             cudaStream_t stream) {
    constexpr size_t ENQ_MAX_TERMS = 2048;
    if (nterms > ENQ_MAX_TERMS)
        return set_error(SV_ERR_ARG, "expectation: at most 2048 terms per call");
    if (nterms == 0) {
        SV_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double), stream));
        return SV_OK;
    }
    uint16_t order[ENQ_MAX_TERMS];
    for (size_t i = 0; i < nterms; ++i) {          // stable insertion sort by X-part
        size_t j = i;
        while (j > 0 && x[order[j - 1]] > x[i]) {
            order[j] = order[j - 1];
            --j;
        }
        order[j] = (uint16_t)i;
    }
    size_t nbatches = 0;
    for (size_t i = 0, run = 0; i < nterms; ++i) {
        run = (i > 0 && x[order[i]] == x[order[i - 1]]) ? run + 1 : 0;
        if (run % svk::EXP_MAX_TERMS == 0) ++nbatches;
    }
    if (nbatches * (size_t)nb_fixed > scratch_doubles)
        return set_error(SV_ERR_ARG, "expectation: too many term batches for the scratch array");
    size_t i = 0, b = 0;
    while (i < nterms) {
        svk::ExpectArgs a;
        std::memset(&a, 0, sizeof(a));
        a.x = x[order[i]];
        while (i < nterms && x[order[i]] == a.x && a.nterms < svk::EXP_MAX_TERMS) {
            const size_t t = order[i++];
            const int y = __builtin_popcountll(a.x & z[t]) & 3;
            const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
            a.z[a.nterms] = z[t];
            a.ccr[a.nterms] = c[t] * re[y];
            a.cci[a.nterms] = c[t] * im[y];
            ++a.nterms;
        }
        a.hb = a.x ? 63 - __builtin_clzll(a.x) : 0;
        a.npairs = a.x ? (1ull << (n - 1)) : (1ull << n);
        double *part = scratch + (b++) * (size_t)nb_fixed;
        if (dtype == SV_C64)
            svk::expect_kernel<float><<<nb_fixed, svk::RED_THREADS, 0, stream>>>(a, psi, part);
        else
            svk::expect_kernel<double><<<nb_fixed, svk::RED_THREADS, 0, stream>>>(a, psi, part);
        SV_CUDA(cudaGetLastError());
    }
    svk::sum_partials<<<1, svk::RED_THREADS, 0, stream>>>(scratch, (int)(nbatches * nb_fixed),
                                                          out_dev);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

sv_status launch_widen(sv_state *s, const void *src_c64, void *dst_c128) {
    const unsigned long long N = 1ull << s->n;
    svk::widen_kernel<<<s->num_sms * 8, 256, 0, s->stream>>>(
        reinterpret_cast<const float2 *>(src_c64), reinterpret_cast<double2 *>(dst_c128), N);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

sv_status launch_set_one(sv_state *s, uint64_t x) {
    svk::set_amp_one<<<1, 1, 0, s->stream>>>(s->buf, x, s->dtype == SV_C128);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

}  // namespace svi
