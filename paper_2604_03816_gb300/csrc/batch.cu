// Batched execution: many states of one width, each with its own circuit, where all the
// circuits share one fused structure (the same targets gate by gate -- a parameter sweep
// of one circuit family fused with the same width).
//
// Layout: the `count` states lie back to back (state i at amplitude offset i * 2^n); the
// per-state matrices of fused gate g lie in a device table [g][state][2 * 4^k].
// Execution: the states are processed in chunks small enough to stay resident in L2;
// for each chunk every fused gate is one launch of a persistent tile kernel that strides
// over all tiles of the chunk's states (the tile geometry is the one of the single-state
// kernels: TMA 1-D bulk staging of 2^h segments, one HBM/L2 read + write per gate;
// complex64 gates of width 4 and 5 run on the tensor-core kernel of apply_tc.cu).  The
// whole launch sequence is captured once into a CUDA graph and replayed while the batch
// object, the chunk size and the fused structure stay the same; only the matrix table is
// refreshed (an H2D copy before the replay).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <system_error>
#include <thread>

#include "plan.h"
#include "ptx.cuh"
#include "sv_internal.h"

namespace svk {

template <typename R> struct BC2;
template <> struct BC2<float> { using T = float2; };
template <> struct BC2<double> { using T = double2; };

__device__ __forceinline__ float bfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double bfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 bmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 bmk(double a, double b) { return make_double2(a, b); }

template <int K>
struct BatchArgs {
    const void *utab;                // [states][2 * 4^K] in the state's precision
    void *psi;                       // first state of the chunk
    int *err;
    unsigned long long tiles_per_state;
    unsigned long long ntiles;       // states * tiles_per_state
    uint32_t n;                      // qubits per state (stride 2^n amplitudes)
    uint32_t L, h;
    uint32_t hi[SV_MAX_K];
    uint32_t lp[K];
};

template <typename R, int K>
__global__ void __launch_bounds__(256) apply_batch_tile(const __grid_constant__ BatchArgs<K> a) {
    using C = typename BC2<R>::T;
    constexpr int D = 1 << K;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ __align__(16) R su[2 * D * D];
    C *tile = reinterpret_cast<C *>(smem);
    const uint32_t seg_amps = 1u << a.L;
    const uint32_t seg_bytes = seg_amps * (uint32_t)sizeof(C);
    const uint32_t nseg = 1u << a.h;
    const uint32_t ngroups = 1u << (a.L + a.h - K);
    const uint32_t barp = smem_u32(&bar);
    uint32_t coff[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((c >> j) & 1) o |= 1u << a.lp[j];
        coff[c] = o;
    }
    SegLanes sl;
    sl.init(a.L, a.h, a.hi, threadIdx.x & 31u);
    if (threadIdx.x == 0) {
        mbar_init(barp, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;
    unsigned long long cur_state = ~0ull;
    // contiguous ranges of tiles per CTA, so that a CTA changes state (and matrix) rarely
    const unsigned long long per_cta = (a.ntiles + gridDim.x - 1) / gridDim.x;
    const unsigned long long t0 = blockIdx.x * per_cta;
    const unsigned long long t1 = min(a.ntiles, t0 + per_cta);
    for (unsigned long long T = t0; T < t1; ++T) {
        const unsigned long long st = T / a.tiles_per_state, t = T % a.tiles_per_state;
        C *psi = reinterpret_cast<C *>(a.psi) + (st << a.n);
        if (st != cur_state) {
            const R *src = reinterpret_cast<const R *>(a.utab) + st * (2ull * D * D);
            for (int i = threadIdx.x; i < 2 * D * D; i += blockDim.x) su[i] = src[i];
            cur_state = st;
        }
        const unsigned long long base = sl.base(t);
        if (threadIdx.x < 32) {                 // warp 0: lane i copies segment i
            if (threadIdx.x == 0) mbar_arrive_expect_tx(barp, seg_bytes * nseg);
            __syncwarp();
            if (threadIdx.x < nseg)
                bulk_g2s(smem_u32(tile + (size_t)threadIdx.x * seg_amps), psi + base + sl.my_off,
                         seg_bytes, barp);
        }
        const bool ok = mbar_wait_bounded(barp, parity);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(a.err, 4);
            if (threadIdx.x < 32) bulk_wait_all();
            return;
        }
        parity ^= 1u;
        for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
            uint32_t b = g;
#pragma unroll
            for (int j = 0; j < K; ++j) b = insert_zero32(b, a.lp[j]);
            C v[D];
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = tile[b | coff[c]];
            // rows: fully unrolled for small gates; for k >= 4 a rolled loop (the matrix
            // comes from shared memory either way) keeps the register count down
#pragma unroll(K <= 3 ? D : 1)
            for (int r = 0; r < D; ++r) {
                R re = 0, im = 0;
                const R *ur_row = su + 2 * r * D;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const R ur = ur_row[2 * c], ui = ur_row[2 * c + 1];
                    re = bfma(ur, v[c].x, re);
                    re = bfma(-ui, v[c].y, re);
                    im = bfma(ur, v[c].y, im);
                    im = bfma(ui, v[c].x, im);
                }
                uint32_t off = b;
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if ((r >> j) & 1) off |= 1u << a.lp[j];
                tile[off] = bmk(re, im);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x < 32) {
            if (threadIdx.x < nseg)
                bulk_s2g(psi + base + sl.my_off, smem_u32(tile + (size_t)threadIdx.x * seg_amps), seg_bytes);
            bulk_commit();
            bulk_wait_read_all();
        }
        __syncthreads();
    }
    if (threadIdx.x < 32) bulk_wait_all();
}

template <typename R, int K>
constexpr uint32_t batch_tile_bits() {
    return sizeof(R) == 4 ? 12u : 11u;
}

// Tile sizes the batched CUDA-core kernel accepts (2^TB amplitudes per CTA); the
// autotuner may pick any of them per batch.
constexpr uint32_t BATCH_TB_MIN = 10, BATCH_TB_MAX = 13;

template <typename R, int K>
struct BatchKernel {
    // The dynamic shared-memory limit is set for the largest tile once; the resident CTAs
    // per SM are measured per tile size.
    static cudaError_t prepare(uint32_t tb, int *blocks_per_sm) {
        static std::once_flag once;
        static int bps[BATCH_TB_MAX + 1] = {};
        static cudaError_t err = cudaSuccess;
        std::call_once(once, [] {
            using C = typename BC2<R>::T;
            err = cudaFuncSetAttribute(apply_batch_tile<R, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int((1u << BATCH_TB_MAX) * sizeof(C)));
            for (uint32_t t = BATCH_TB_MIN; t <= BATCH_TB_MAX && err == cudaSuccess; ++t) {
                err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[t], apply_batch_tile<R, K>, 256,
                                                                    int((1u << t) * sizeof(C)));
                if (bps[t] < 1) bps[t] = 1;
            }
        });
        *blocks_per_sm = bps[tb];
        return err;
    }
    static sv_status launch(const sv_batch_launch &L) {
        using C = typename BC2<R>::T;
        const uint32_t tb = L.tile_bits ? L.tile_bits : batch_tile_bits<R, K>();
        int bps = 1;
        const cudaError_t e = prepare(tb, &bps);
        if (e != cudaSuccess)
            return svi::set_error(SV_ERR_CUDA, std::string("batch kernel setup: ") + cudaGetErrorString(e));
        const Plan p = make_plan(L.n, K, L.t, tb);
        BatchArgs<K> a;
        a.utab = L.utab;
        a.psi = L.psi;
        a.err = L.err;
        a.tiles_per_state = p.ntiles;
        a.ntiles = p.ntiles * L.states;
        a.n = L.n;
        a.L = p.L;
        a.h = p.h;
        for (int j = 0; j < SV_MAX_K; ++j) a.hi[j] = p.hi[j];
        for (int j = 0; j < K; ++j) a.lp[j] = p.lp[j];
        const unsigned long long cap = (unsigned long long)bps * L.num_sms;
        const unsigned grid = (unsigned)std::min<unsigned long long>(a.ntiles, cap);
        const size_t bytes = (size_t(1) << (p.L + p.h)) * sizeof(C);
        apply_batch_tile<R, K><<<grid, 256, bytes, L.stream>>>(a);
        SV_CUDA(cudaGetLastError());
        return SV_OK;
    }
};

// ---------------------------------------------------------------- batched expectation

constexpr int BEXP_TERMS = 32;
constexpr int BEXP_BLOCKS = 16;     // blocks per state

struct BatchExpectArgs {
    unsigned long long x;
    unsigned long long z[BEXP_TERMS];
    double ccr[BEXP_TERMS], cci[BEXP_TERMS];
    int nterms, hb;
    unsigned long long npairs;
    uint32_t n;
};

__device__ __forceinline__ float bprob(float x, float y) { return __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)); }
__device__ __forceinline__ double bprob(double x, double y) { return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)); }

// grid (BEXP_BLOCKS, states): partial[state * BEXP_BLOCKS + block]
template <typename R>
__global__ void batch_expect_kernel(const __grid_constant__ BatchExpectArgs a, const void *psi_,
                                    double *partial) {
    using C = typename BC2<R>::T;
    const C *psi = reinterpret_cast<const C *>(psi_) + ((unsigned long long)blockIdx.y << a.n);
    double acc = 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // Z-only terms: runs of eight consecutive amplitudes per thread, the term weights and
    // the run's sum in the state's precision (FP32 for complex64: GB300's FP64 pipe is
    // narrow), one FP64 add per run
    __shared__ R cw[BEXP_TERMS];
    if (threadIdx.x < BEXP_TERMS) cw[threadIdx.x] = (R)a.ccr[threadIdx.x];
    __syncthreads();
    const unsigned long long nrun = a.x == 0 ? a.npairs / 8 : 0;
    for (unsigned long long r = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrun;
         r += stride) {
        C v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = psi[r * 8 + q];
        // terms outside, the eight amplitudes inside: eight independent weight sums
        R w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = 0;
        for (int t = 0; t < a.nterms; ++t) {
            const unsigned long long z = a.z[t];
            const R c = cw[t];
            const int hi = __popcll((r * 8) & z);
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q] += ((hi + __popc((uint32_t)q & (uint32_t)z)) & 1) ? -c : c;
        }
        R run = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) run += w[q] * bprob(v[q].x, v[q].y);
        acc += (double)run;
    }
    for (unsigned long long i = nrun * 8 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         i < a.npairs; i += stride) {
        if (a.x == 0) {
            const C v = psi[i];
            double w = 0.0;
            for (int t = 0; t < a.nterms; ++t) w += (__popcll(i & a.z[t]) & 1) ? -a.ccr[t] : a.ccr[t];
            acc += w * (double)bprob(v.x, v.y);
        } else {
            const unsigned long long k = insert_zero64(i, (uint32_t)a.hb), k2 = k ^ a.x;
            const C p = psi[k], q = psi[k2];
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
            acc += re * w1r - im * w1i + re * w2r + im * w2i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += ws[w];
        partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = r;
    }
}

__global__ void batch_set_one(void *psi, unsigned long long x, uint32_t n, uint32_t count, int is_c128) {
    const uint32_t st = blockIdx.x * blockDim.x + threadIdx.x;
    if (st >= count) return;
    const unsigned long long idx = ((unsigned long long)st << n) + x;
    if (is_c128) reinterpret_cast<double2 *>(psi)[idx] = make_double2(1.0, 0.0);
    else reinterpret_cast<float2 *>(psi)[idx] = make_float2(1.f, 0.f);
}

// out[state] += sum of that state's partials (fixed order)
__global__ void batch_sum_partials(const double *partial, int per_state, int states, double *out) {
    const int st = blockIdx.x * blockDim.x + threadIdx.x;
    if (st >= states) return;
    double r = 0.0;
    for (int b = 0; b < per_state; ++b) r += partial[(size_t)st * per_state + b];
    out[st] += r;
}

}  // namespace svk

// ------------------------------------------------------------------ batch object

struct sv_batch {
    uint32_t n = 0, count = 0;
    sv_dtype dtype = SV_C64;
    void *buf = nullptr;
    size_t cap = 0;
    bool owned = false;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int *err = nullptr;                 // device error word
    double *partial = nullptr;          // count * BEXP_BLOCKS
    double *results = nullptr;          // count
    void *utab = nullptr;               // device matrix table
    size_t utab_cap = 0;
    void *utab_host = nullptr;          // pinned staging of the table
    size_t utab_host_cap = 0;
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture the graph
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t staged = nullptr;       // the last H2D copy out of utab_host has finished
    bool staged_pending = false;
};

namespace svi {

static size_t elem_bytes_b(sv_dtype d) { return d == SV_C64 ? 8 : 16; }

static sv_status batch_launch(const sv_batch_launch &L) {
    if (L.tc) return svk::launch_tc_batch(L);
    if (L.dtype == SV_C64) {
        switch (L.k) {
            case 1: return svk::BatchKernel<float, 1>::launch(L);
            case 2: return svk::BatchKernel<float, 2>::launch(L);
            case 3: return svk::BatchKernel<float, 3>::launch(L);
            case 4: return svk::BatchKernel<float, 4>::launch(L);
            default: return svk::BatchKernel<float, 5>::launch(L);
        }
    }
    switch (L.k) {
        case 1: return svk::BatchKernel<double, 1>::launch(L);
        case 2: return svk::BatchKernel<double, 2>::launch(L);
        case 3: return svk::BatchKernel<double, 3>::launch(L);
        case 4: return svk::BatchKernel<double, 4>::launch(L);
        default: return svk::BatchKernel<double, 5>::launch(L);
    }
}

static cudaError_t batch_prepare(sv_dtype dt, uint32_t k) {
    int bps = 0;
    if (dt == SV_C64) {
        switch (k) {
            case 1: return svk::BatchKernel<float, 1>::prepare(svk::BATCH_TB_MAX, &bps);
            case 2: return svk::BatchKernel<float, 2>::prepare(svk::BATCH_TB_MAX, &bps);
            case 3: return svk::BatchKernel<float, 3>::prepare(svk::BATCH_TB_MAX, &bps);
            case 4: return svk::BatchKernel<float, 4>::prepare(svk::BATCH_TB_MAX, &bps);
            default: return svk::BatchKernel<float, 5>::prepare(svk::BATCH_TB_MAX, &bps);
        }
    }
    switch (k) {
        case 1: return svk::BatchKernel<double, 1>::prepare(svk::BATCH_TB_MAX, &bps);
        case 2: return svk::BatchKernel<double, 2>::prepare(svk::BATCH_TB_MAX, &bps);
        case 3: return svk::BatchKernel<double, 3>::prepare(svk::BATCH_TB_MAX, &bps);
        case 4: return svk::BatchKernel<double, 4>::prepare(svk::BATCH_TB_MAX, &bps);
        default: return svk::BatchKernel<double, 5>::prepare(svk::BATCH_TB_MAX, &bps);
    }
}

}  // namespace svi

using namespace svi;

extern "C" {

sv_status sv_batch_alloc(uint32_t n, sv_dtype dtype, uint32_t count, void *dev_buf, size_t bytes,
                         void *stream, sv_batch **out) {
    clear_error();
    if (!out) return set_error(SV_ERR_ARG, "sv_batch_alloc: null out");
    *out = nullptr;
    if (n < 1 || n > SV_MAX_QUBITS) return set_error(SV_ERR_ARG, "sv_batch_alloc: n must be 1..34");
    if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "sv_batch_alloc: bad dtype");
    if (count < 1 || count > 65535) return set_error(SV_ERR_ARG, "sv_batch_alloc: count must be 1..65535");
    const size_t need = (elem_bytes_b(dtype) << n) * count;
    if (dev_buf && bytes < need) return set_error(SV_ERR_ARG, "sv_batch_alloc: buffer too small");
    if (dev_buf && (reinterpret_cast<uintptr_t>(dev_buf) & 15u))
        return set_error(SV_ERR_ARG, "sv_batch_alloc: buffer must be 16-byte aligned");
    sv_batch *b = new (std::nothrow) sv_batch();
    if (!b) return set_error(SV_ERR_OOM, "sv_batch_alloc: host allocation failed");
    b->n = n;
    b->count = count;
    b->dtype = dtype;
    b->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) {
        if (dev_buf) {
            b->buf = dev_buf;
            b->cap = bytes;
        } else {
            e = cudaMalloc(&b->buf, need);
            b->cap = need;
            b->owned = true;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->err), 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, 256, b->stream);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&b->partial), sizeof(double) * count * svk::BEXP_BLOCKS);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->results), sizeof(double) * count);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        const std::string msg = std::string("sv_batch_alloc: ") + cudaGetErrorString(e);
        sv_batch_free(b);
        return set_error(SV_ERR_OOM, msg);
    }
    sv_status st = sv_batch_set_basis(b, 0);
    if (st != SV_OK) {
        sv_batch_free(b);
        return st;
    }
    *out = b;
    return SV_OK;
}

sv_status sv_batch_free(sv_batch *b) {
    if (!b) return SV_OK;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->owned && b->buf) cudaFree(b->buf);
    if (b->err) cudaFree(b->err);
    if (b->partial) cudaFree(b->partial);
    if (b->results) cudaFree(b->results);
    if (b->utab) cudaFree(b->utab);
    if (b->utab_host) cudaFreeHost(b->utab_host);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->staged) cudaEventDestroy(b->staged);
    delete b;
    return SV_OK;
}

sv_status sv_batch_set_basis(sv_batch *b, uint64_t x) {
    clear_error();
    if (!b) return set_error(SV_ERR_ARG, "sv_batch_set_basis: null batch");
    if (x >> b->n) return set_error(SV_ERR_ARG, "sv_batch_set_basis: x >= 2^n");
    const size_t sb = elem_bytes_b(b->dtype) << b->n;
    SV_CUDA(cudaMemsetAsync(b->buf, 0, sb * b->count, b->stream));
    svk::batch_set_one<<<(b->count + 127) / 128, 128, 0, b->stream>>>(b->buf, x, b->n, b->count,
                                                                      b->dtype == SV_C128);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

sv_status sv_batch_get_state(sv_batch *b, uint32_t i, void *dst, int dst_on_device) {
    clear_error();
    if (!b || !dst || i >= b->count) return set_error(SV_ERR_ARG, "sv_batch_get_state: bad argument");
    const size_t sb = elem_bytes_b(b->dtype) << b->n;
    SV_CUDA(cudaMemcpyAsync(dst, static_cast<char *>(b->buf) + sb * i, sb,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    if (!dst_on_device) SV_CUDA(cudaStreamSynchronize(b->stream));
    return SV_OK;
}

sv_status sv_batch_apply(sv_batch *b, const sv_circuit *const *circuits, const sv_batch_opts *opts,
                         sv_batch_report *rep) {
    clear_error();
    if (!b || !circuits) return set_error(SV_ERR_ARG, "sv_batch_apply: null argument");
    const sv_circuit *c0 = circuits[0];
    if (!c0) return set_error(SV_ERR_ARG, "sv_batch_apply: null circuit");
    if (c0->n != b->n) return set_error(SV_ERR_ARG, "sv_batch_apply: circuit built for another n");
    const size_t G = c0->gates.size();
    for (uint32_t i = 1; i < b->count; ++i) {
        const sv_circuit *c = circuits[i];
        if (!c || c->n != b->n || c->gates.size() != G)
            return set_error(SV_ERR_ARG, "sv_batch_apply: circuit " + std::to_string(i) +
                                             " does not share the fused structure");
        for (size_t g = 0; g < G; ++g) {
            const Gate &a = c0->gates[g], &z = c->gates[g];
            if (a.k != z.k || std::memcmp(a.t, z.t, sizeof(a.t)) != 0)
                return set_error(SV_ERR_ARG, "sv_batch_apply: circuit " + std::to_string(i) +
                                                 " differs in the targets of fused gate " +
                                                 std::to_string(g));
        }
    }
    const size_t eb = b->dtype == SV_C64 ? 4 : 8;   // bytes of one real
    std::vector<size_t> goff(G + 1, 0);
    for (size_t g = 0; g < G; ++g)
        goff[g + 1] = goff[g] + (size_t)b->count * 2 * ((size_t)1 << (2 * c0->gates[g].k)) * eb;
    const size_t tab = goff[G];
    if (tab > b->utab_host_cap) {
        if (b->utab_host) cudaFreeHost(b->utab_host);
        b->utab_host = nullptr;
        b->utab_host_cap = 0;
        SV_CUDA(cudaStreamSynchronize(b->stream));
        SV_CUDA(cudaMallocHost(&b->utab_host, tab));
        b->utab_host_cap = tab;
    }
    if (tab > b->utab_cap) {
        SV_CUDA(cudaStreamSynchronize(b->stream));
        if (b->utab) cudaFree(b->utab);
        b->utab = nullptr;
        b->utab_cap = 0;
        SV_CUDA(cudaMalloc(&b->utab, tab));
        b->utab_cap = tab;
        if (b->graph) {                 // the graph holds the old table address
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            b->graph_key.clear();
        }
    }
    if (b->staged_pending) SV_CUDA(cudaEventSynchronize(b->staged));   // staging buffer is free
    // the table [gate][state][2 4^k] in the state's precision, states split over host threads
    auto fill = [&](uint32_t i0, uint32_t i1) {
        for (size_t g = 0; g < G; ++g) {
            const size_t d2 = (size_t)1 << (2 * c0->gates[g].k);
            char *dst = static_cast<char *>(b->utab_host) + goff[g];
            for (uint32_t i = i0; i < i1; ++i) {
                const std::vector<cplx> &u = circuits[i]->gates[g].u;
                if (b->dtype == SV_C64) {
                    float *f = reinterpret_cast<float *>(dst) + (size_t)i * 2 * d2;
                    for (size_t e = 0; e < d2; ++e) {
                        f[2 * e] = (float)u[e].real();
                        f[2 * e + 1] = (float)u[e].imag();
                    }
                } else {
                    double *f = reinterpret_cast<double *>(dst) + (size_t)i * 2 * d2;
                    for (size_t e = 0; e < d2; ++e) {
                        f[2 * e] = u[e].real();
                        f[2 * e + 1] = u[e].imag();
                    }
                }
            }
        }
    };
    {
        const size_t work = tab / 4;                      // entries to convert, roughly
        const uint32_t hw = std::max(1u, std::thread::hardware_concurrency());
        const uint32_t nt = (uint32_t)std::min<size_t>({(size_t)std::min(hw, 16u), (size_t)b->count,
                                                        std::max<size_t>(1, work >> 18)});
        std::vector<std::thread> th;
        const uint32_t per = (b->count + nt - 1) / nt;
        try {
            for (uint32_t w = 1; w < nt; ++w) {
                const uint32_t i0 = std::min(b->count, w * per), i1 = std::min(b->count, i0 + per);
                if (i0 < i1) th.emplace_back(fill, i0, i1);
            }
        } catch (const std::system_error &) {
            // no more threads: the calling thread fills the rest below
        }
        const uint32_t done_by_threads = (uint32_t)th.size();
        fill(0, std::min(b->count, per));
        for (uint32_t w = done_by_threads + 1; w < nt; ++w) {
            const uint32_t i0 = std::min(b->count, w * per), i1 = std::min(b->count, i0 + per);
            if (i0 < i1) fill(i0, i1);
        }
        for (std::thread &t : th) t.join();
    }
    SV_CUDA(cudaMemcpyAsync(b->utab, b->utab_host, tab, cudaMemcpyHostToDevice, b->stream));
    SV_CUDA(cudaEventRecord(b->staged, b->stream));
    b->staged_pending = true;

    const size_t sbytes = elem_bytes_b(b->dtype) << b->n;
    size_t l2 = opts && opts->l2_bytes ? opts->l2_bytes : (size_t(64) << 20);
    uint32_t chunk = opts && opts->chunk_states ? opts->chunk_states
                                                 : (uint32_t)std::max<size_t>(1, l2 / sbytes);
    chunk = std::min(chunk, b->count);
    const bool use_graph = !(opts && opts->no_graph);
    const bool timing = opts && opts->timing;
    const uint32_t tile_bits = opts ? opts->tile_bits : 0u;
    if (tile_bits && (tile_bits < svk::BATCH_TB_MIN || tile_bits > svk::BATCH_TB_MAX))
        return set_error(SV_ERR_ARG, "sv_batch_apply: tile_bits must be 0 or 10..13");
    // complex64 gates of width 4 and 5 on the tensor cores (states of at least 12 qubits)
    const bool tc_ok = b->dtype == SV_C64 && b->n >= 12 && !(opts && opts->no_tensor_cores);
    auto use_tc = [&](const Gate &g) { return tc_ok && (g.k == 4 || g.k == 5); };

    std::string key = std::to_string(b->n) + "/" + std::to_string(b->count) + "/" +
                      std::to_string(b->dtype) + "/" + std::to_string(chunk) + "/" +
                      (tc_ok ? "tc/" : "cc/") + std::to_string(tile_bits) + "/";
    for (const Gate &g : c0->gates)
        for (uint32_t j = 0; j < g.k; ++j) key += std::to_string(g.t[j]) + (j + 1 < g.k ? "," : ";");

    auto enqueue_all = [&](cudaStream_t stream) -> sv_status {
        for (uint32_t s0 = 0; s0 < b->count; s0 += chunk) {
            const uint32_t ns = std::min(chunk, b->count - s0);
            for (size_t g = 0; g < G; ++g) {
                const Gate &gg = c0->gates[g];
                sv_batch_launch L;
                L.dtype = b->dtype;
                L.k = gg.k;
                L.n = b->n;
                for (uint32_t j = 0; j < SV_MAX_K; ++j) L.t[j] = gg.t[j];
                L.states = ns;
                L.psi = static_cast<char *>(b->buf) + sbytes * s0;
                L.utab = static_cast<char *>(b->utab) + goff[g] +
                         (size_t)s0 * 2 * ((size_t)1 << (2 * gg.k)) * eb;
                L.err = b->err;
                L.stream = stream;
                L.num_sms = b->num_sms;
                L.tc = use_tc(gg);
                L.tile_bits = tile_bits;
                sv_status st = batch_launch(L);
                if (st != SV_OK) return st;
            }
        }
        return SV_OK;
    };

    sv_batch_report r;
    std::memset(&r, 0, sizeof(r));
    r.chunk_states = chunk;
    r.tile_bits = tile_bits ? tile_bits : (b->dtype == SV_C64 ? 12u : 11u);
    r.passes = (uint64_t)G * b->count;
    r.launches = (uint64_t)G * ((b->count + chunk - 1) / chunk);
    r.bytes = (uint64_t)G * b->count * 2ull * sbytes;
    if (timing) SV_CUDA(cudaEventRecord(b->ev0, b->stream));
    if (!use_graph) {
        sv_status st = enqueue_all(b->stream);
        if (st != SV_OK) return st;
    } else {
        if (!b->graph || b->graph_key != key) {
            for (const Gate &g : c0->gates) SV_CUDA(use_tc(g) ? svk::tc_batch_prepare() : batch_prepare(b->dtype, g.k));
            if (b->graph) {
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
            cudaGraph_t graph = nullptr;
            // captured on a private stream (the caller's may be the legacy default stream,
            // which cannot be captured); the graph is then launched on the caller's stream
            SV_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            sv_status st = enqueue_all(b->cap_stream);
            cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
            if (st != SV_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) return set_error(SV_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->graph = nullptr;
                return set_error(SV_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            }
            b->graph_key = key;
        } else {
            r.graph_reused = 1;
        }
        SV_CUDA(cudaGraphLaunch(b->graph, b->stream));
    }
    if (timing) {
        SV_CUDA(cudaEventRecord(b->ev1, b->stream));
        SV_CUDA(cudaEventSynchronize(b->ev1));
        float ms = 0.f;
        SV_CUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        r.apply_ms = ms;
    }
    if (rep) *rep = r;
    return SV_OK;
}

sv_status sv_batch_expect(sv_batch *b, const uint64_t *xmask, const uint64_t *zmask, const double *coef,
                          size_t nterms, double *out) {
    clear_error();
    if (!b || !out || (nterms && (!xmask || !zmask || !coef)))
        return set_error(SV_ERR_ARG, "sv_batch_expect: null argument");
    const uint64_t lim = (1ull << b->n) - 1;
    for (size_t t = 0; t < nterms; ++t)
        if ((xmask[t] & ~lim) || (zmask[t] & ~lim))
            return set_error(SV_ERR_ARG, "sv_batch_expect: Pauli mask names a qubit >= n");
    SV_CUDA(cudaMemsetAsync(b->results, 0, sizeof(double) * b->count, b->stream));
    std::vector<size_t> order(nterms);
    for (size_t i = 0; i < nterms; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return xmask[a] < xmask[c]; });
    size_t i = 0;
    while (i < nterms) {
        svk::BatchExpectArgs a;
        std::memset(&a, 0, sizeof(a));
        a.x = xmask[order[i]];
        while (i < nterms && xmask[order[i]] == a.x && a.nterms < svk::BEXP_TERMS) {
            const size_t t = order[i++];
            const int y = __builtin_popcountll(a.x & zmask[t]) & 3;
            const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
            a.z[a.nterms] = zmask[t];
            a.ccr[a.nterms] = coef[t] * re[y];
            a.cci[a.nterms] = coef[t] * im[y];
            ++a.nterms;
        }
        a.hb = a.x ? 63 - __builtin_clzll(a.x) : 0;
        a.npairs = a.x ? (1ull << (b->n - 1)) : (1ull << b->n);
        a.n = b->n;
        const dim3 grid(svk::BEXP_BLOCKS, b->count);
        if (b->dtype == SV_C64)
            svk::batch_expect_kernel<float><<<grid, 256, 0, b->stream>>>(a, b->buf, b->partial);
        else
            svk::batch_expect_kernel<double><<<grid, 256, 0, b->stream>>>(a, b->buf, b->partial);
        SV_CUDA(cudaGetLastError());
        svk::batch_sum_partials<<<(b->count + 127) / 128, 128, 0, b->stream>>>(
            b->partial, svk::BEXP_BLOCKS, (int)b->count, b->results);
        SV_CUDA(cudaGetLastError());
    }
    SV_CUDA(cudaMemcpyAsync(out, b->results, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream));
    SV_CUDA(cudaStreamSynchronize(b->stream));
    int err = 0;
    SV_CUDA(cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        SV_CUDA(cudaMemset(b->err, 0, sizeof(int)));
        return set_error(SV_ERR_TIMEOUT, "a bounded device-side wait gave up in a batched pass");
    }
    return SV_OK;
}

sv_status sv_batch_tune(sv_batch *b, const sv_gate *gates, size_t ngates, uint32_t kmin, uint32_t kmax,
                        sv_tune_result *out) {
    clear_error();
    if (!b || !out || (ngates && !gates)) return set_error(SV_ERR_ARG, "sv_batch_tune: null argument");
    if (kmin < 1 || kmax > SV_MAX_K || kmin > kmax)
        return set_error(SV_ERR_ARG, "sv_batch_tune: need 1 <= kmin <= kmax <= 5");
    // cache key: batch shape + the target sequence of the gates (Algorithm 1's idea of
    // measuring once and caching, applied to the fusion width and the chunk size)
    std::string key = std::to_string(b->n) + "/" + std::to_string(b->count) + "/" +
                      std::to_string(b->dtype) + "/" + std::to_string(kmin) + "-" + std::to_string(kmax) + "/";
    for (size_t i = 0; i < ngates; ++i) {
        if (gates[i].k < 1 || gates[i].k > SV_MAX_K) return set_error(SV_ERR_ARG, "sv_batch_tune: bad gate");
        for (uint32_t j = 0; j < gates[i].k; ++j) key += std::to_string(gates[i].targets[j]) + ",";
        key += ";";
    }
    static std::mutex mu;
    static std::map<std::string, sv_tune_result> cache;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *out = it->second;
            out->cached = 1;
            return SV_OK;
        }
    }
    sv_tune_result r;
    std::memset(&r, 0, sizeof(r));
    double best = 1e300;
    // chunk budgets: L2-resident chunks suit the CUDA-core passes; the tensor-core passes
    // (a fixed cost of about 20 us per launch) prefer few large launches
    const size_t sbytes = (b->dtype == SV_C64 ? size_t(8) : size_t(16)) << b->n;
    const size_t l2s[3] = {size_t(64) << 20, size_t(512) << 20, sbytes * b->count};
    const bool tc_ok = b->dtype == SV_C64 && b->n >= 12;
    for (uint32_t k = kmin; k <= kmax; ++k) {
        sv_circuit *c = nullptr;
        sv_status st = sv_fuse(gates, ngates, b->n, k, &c);
        if (st != SV_OK) return st;
        std::vector<const sv_circuit *> cs(b->count, c);
        double kbest = 1e300;
        size_t kl2 = l2s[0];
        auto time_it = [&](size_t l2, uint32_t tb) -> double {
            sv_batch_opts o;
            std::memset(&o, 0, sizeof(o));
            o.l2_bytes = l2;
            o.timing = 1;
            o.tile_bits = tb;
            sv_batch_report rep;
            double ms = 1e300;
            for (int rep_i = 0; rep_i < 3 && st == SV_OK; ++rep_i) {   // first run warms up
                st = sv_batch_apply(b, cs.data(), &o, &rep);
                if (rep_i > 0) ms = std::min(ms, rep.apply_ms);
            }
            if (st == SV_OK && ms < best) {
                best = ms;
                r.best_k = k;
                r.l2_bytes = l2;
                r.tile_bits = tb;
            }
            return ms;
        };
        for (size_t l2 : l2s) {
            const double ms = time_it(l2, 0);
            if (st != SV_OK) break;
            if (ms < kbest) {
                kbest = ms;
                kl2 = l2;
            }
        }
        // the tile size of the CUDA-core passes, at this width's best chunking, when the
        // schedule has such passes (complex128, narrow gates, tensor cores not eligible)
        bool cuda_core = false;
        for (const Gate &g : c->gates) cuda_core = cuda_core || !(tc_ok && (g.k == 4 || g.k == 5));
        if (cuda_core && st == SV_OK)
            for (uint32_t tb = svk::BATCH_TB_MIN; tb <= svk::BATCH_TB_MAX && st == SV_OK; ++tb)
                kbest = std::min(kbest, time_it(kl2, tb));
        sv_circuit_free(c);
        if (st != SV_OK) return st;
        r.ms[k] = kbest;
    }
    r.best_ms = best;
    {
        std::lock_guard<std::mutex> lock(mu);
        cache[key] = r;
    }
    *out = r;
    return sv_batch_set_basis(b, 0);
}

sv_status sv_batch_sync(sv_batch *b) {
    clear_error();
    if (!b) return set_error(SV_ERR_ARG, "sv_batch_sync: null batch");
    SV_CUDA(cudaStreamSynchronize(b->stream));
    int err = 0;
    SV_CUDA(cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        SV_CUDA(cudaMemset(b->err, 0, sizeof(int)));
        return set_error(SV_ERR_TIMEOUT, "a bounded device-side wait gave up in a batched pass");
    }
    return SV_OK;
}

}  // extern "C"
