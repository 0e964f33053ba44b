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
        float sa = prob_of(a.x, a.y) + prob_of(a.z, a.w);
        float sb = prob_of(b.x, b.y) + prob_of(b.z, b.w);
        float sc = prob_of(c.x, c.y) + prob_of(c.z, c.w);
        float sd = prob_of(d.x, d.y) + prob_of(d.z, d.w);
        acc += (double)sa + (double)sb + (double)sc + (double)sd;
    }
    for (; i < nvec; i += stride) {
        float4 a = v[i];
        acc += (double)(prob_of(a.x, a.y) + prob_of(a.z, a.w));
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

// ---------------------------------------------------------------- top-k

// (p, idx) order: larger p first, then smaller index.
__device__ __forceinline__ bool better(double pa, unsigned long long ia, double pb,
                                       unsigned long long ib) {
    return pa > pb || (pa == pb && ia < ib);
}

struct TopList {   // one warp's 64 entries, two per lane, plus the current worst
    double p0, p1;
    unsigned long long i0, i1;
    double wp;
    unsigned long long wi;
    int wl, ws;    // lane and slot of the worst entry

    __device__ void init() {
        p0 = p1 = -1.0;
        i0 = i1 = ~0ull;
        find_worst();
    }
    __device__ void find_worst() {
        const int lane = threadIdx.x & 31;
        // this lane's worse entry
        bool second = better(p0, i0, p1, i1);
        double p = second ? p1 : p0;
        unsigned long long ix = second ? i1 : i0;
        int l = lane, s = second ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double op = __shfl_xor_sync(0xffffffffu, p, o);
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
    __device__ void offer(double p, unsigned long long ix, bool valid) {
        const int lane = threadIdx.x & 31;
        unsigned mask = __ballot_sync(0xffffffffu, valid && better(p, ix, wp, wi));
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const double cp = __shfl_sync(0xffffffffu, p, src);
            const unsigned long long ci = __shfl_sync(0xffffffffu, ix, src);
            if (!better(cp, ci, wp, wi)) continue;     // uniform across the warp
            if (lane == wl) {
                if (ws == 0) { p0 = cp; i0 = ci; } else { p1 = cp; i1 = ci; }
            }
            find_worst();
        }
    }
};

template <typename R>
__global__ void topk_pass1(const void *psi_, unsigned long long N, unsigned long long chunk,
                           double *cand_p, unsigned long long *cand_i) {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C *psi = reinterpret_cast<const C *>(psi_);
    const int lane = threadIdx.x & 31;
    const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    TopList L;
    L.init();
    const unsigned long long lo = warp * chunk, hi = min(N, lo + chunk);
    for (unsigned long long b = lo; b < hi; b += 32) {
        const unsigned long long k = b + lane;
        double p = -1.0;
        if (k < hi) {
            const C v = psi[k];
            p = (double)prob_of(v.x, v.y);
        }
        L.offer(p, k, k < hi);
    }
    cand_p[warp * 64 + 2 * lane] = L.p0;
    cand_i[warp * 64 + 2 * lane] = L.i0;
    cand_p[warp * 64 + 2 * lane + 1] = L.p1;
    cand_i[warp * 64 + 2 * lane + 1] = L.i1;
}

// One warp merges m candidates and writes the best 64, sorted.
__global__ void topk_pass2(const double *cand_p, const unsigned long long *cand_i,
                           unsigned long long m, double *out_p, unsigned long long *out_i) {
    __shared__ double sp[64];
    __shared__ unsigned long long si[64];
    const int lane = threadIdx.x & 31;
    TopList L;
    L.init();
    for (unsigned long long b = 0; b < m; b += 32) {
        const unsigned long long j = b + lane;
        const bool ok = j < m;
        L.offer(ok ? cand_p[j] : -1.0, ok ? cand_i[j] : ~0ull, ok && cand_p[ok ? j : 0] >= 0.0);
    }
    sp[2 * lane] = L.p0; si[2 * lane] = L.i0;
    sp[2 * lane + 1] = L.p1; si[2 * lane + 1] = L.i1;
    __syncwarp();
    if (lane == 0) {
        for (int a = 1; a < 64; ++a) {          // insertion sort, best first
            const double p = sp[a];
            const unsigned long long ix = si[a];
            int b = a - 1;
            while (b >= 0 && better(p, ix, sp[b], si[b])) {
                sp[b + 1] = sp[b]; si[b + 1] = si[b];
                --b;
            }
            sp[b + 1] = p; si[b + 1] = ix;
        }
        for (int a = 0; a < 64; ++a) { out_p[a] = sp[a]; out_i[a] = si[a]; }
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
            if (s->dtype == SV_C64)
                svk::expect_kernel<float><<<nb, svk::RED_THREADS, 0, s->stream>>>(a, s->buf, partial);
            else
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
    int blocks = std::min(s->num_sms * 2, TOPK_MAX_WARPS / warps_per_block);
    unsigned long long nwarps = (unsigned long long)blocks * warps_per_block;
    unsigned long long chunk = (N + nwarps - 1) / nwarps;
    chunk = (chunk + 31) / 32 * 32;
    double *cp = reinterpret_cast<double *>(s->ws + WS_TOPK);
    unsigned long long *ci = reinterpret_cast<unsigned long long *>(s->ws + WS_TOPK) + TOPK_MAX_WARPS * 64;
    double *op = reinterpret_cast<double *>(s->ws + WS_TOPK + WS_TOPK_BYTES);
    unsigned long long *oi = reinterpret_cast<unsigned long long *>(op + 64);
    if (s->dtype == SV_C64)
        svk::topk_pass1<float><<<blocks, threads, 0, s->stream>>>(s->buf, N, chunk, cp, ci);
    else
        svk::topk_pass1<double><<<blocks, threads, 0, s->stream>>>(s->buf, N, chunk, cp, ci);
    SV_CUDA(cudaGetLastError());
    svk::topk_pass2<<<1, 32, 0, s->stream>>>(cp, ci, nwarps * 64, op, oi);
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
