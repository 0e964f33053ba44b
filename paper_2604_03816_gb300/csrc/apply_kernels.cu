// Fused-gate application: one HBM read + write pass per dense k-qubit gate (k <= 5).
//
// Semantics (Eq. 3 generalised to k targets, the gate record of Section 3):
//   psi'[i] = sum_c U[loc(i)][c] psi[i with target bits replaced by c],
//   loc(i) = sum_j bit(i, t_j) 2^j,  targets t_0 < ... < t_{k-1}.
//
// Design (sm_103a).  A CTA owns a tile of 2^TB amplitudes: the index bits [0, L) plus
// the h targets that lie at or above L ("high" targets), with L + h = TB.  The tile is
// 2^h contiguous segments of 2^L amplitudes, so it is moved with 2^h 1-D bulk TMA
// copies (cp.async.bulk) into shared memory, completion counted on an mbarrier, and
// written back with bulk stores: every gate costs one coalesced read and one write of
// the state whatever its targets, so no qubit-permutation pass is ever needed.  Inside
// the tile every group of 2^k amplitudes (all tile bits fixed except the targets) is
// gathered into registers, multiplied by U (held in the kernel's parameter space, read
// as constant-bank operands of the FMAs) and scattered back.  c64 computes in FP32,
// c128 in FP64.  A persistent grid (resident CTAs x SMs) strides over the tiles.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "plan.h"
#include "ptx.cuh"
#include "sv_internal.h"

namespace svk {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename R, int K>
struct ApplyArgs {
    R u[2 << (2 * K)];        // 2^K x 2^K complex, row-major interleaved
    void *psi;
    int *err;
    unsigned long long ntiles;
    uint32_t L, h;            // tile = bits [0, L) + h high targets
    uint32_t hi[SV_MAX_K];    // global bit positions of the high targets (ascending)
    uint32_t lp[K];           // local tile positions of all K targets (ascending)
};

template <typename R, int K>
__global__ void __launch_bounds__(256) apply_tile(const __grid_constant__ ApplyArgs<R, K> a) {
    using C = typename C2<R>::T;
    constexpr int D = 1 << K;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar;
    C *tile = reinterpret_cast<C *>(smem);
    C *psi = reinterpret_cast<C *>(a.psi);

    const uint32_t seg_amps = 1u << a.L;
    const uint32_t seg_bytes = seg_amps * (uint32_t)sizeof(C);
    const uint32_t nseg = 1u << a.h;
    const uint32_t ngroups = 1u << (a.L + a.h - K);
    const uint32_t barp = smem_u32(&bar);

    uint32_t coff[D];   // offset of group member c from the group's base
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
    for (unsigned long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
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
            if (threadIdx.x == 0) atomicOr(a.err, 1);
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
                tile[b | coff[r]] = mk(re, im);
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

// Tile bits per (precision, k): 32 KB tiles for k <= 3, larger tiles for k = 4, 5 so
// that every one of the 256 threads owns at least one group.
template <typename R, int K>
constexpr uint32_t tile_bits() {
    return sizeof(R) == 4 ? (K <= 4 ? 12u : 13u) : (K <= 3 ? 11u : (K == 4 ? 12u : 13u));
}

template <typename R, int K>
sv_status launch_apply_t(sv_state *s, const svi::Gate &g) {
    constexpr uint32_t TB = tile_bits<R, K>();
    using C = typename C2<R>::T;
    static std::once_flag once;
    static int blocks_per_sm = 1;
    static cudaError_t init_err = cudaSuccess;
    std::call_once(once, [] {
        const int maxb = int((1u << TB) * sizeof(C));
        init_err = cudaFuncSetAttribute(apply_tile<R, K>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
        if (init_err == cudaSuccess)
            init_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm,
                                                                     apply_tile<R, K>, 256, maxb);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    });
    if (init_err != cudaSuccess)
        return svi::set_error(SV_ERR_CUDA, std::string("apply kernel setup: ") +
                                               cudaGetErrorString(init_err));
    const Plan p = make_plan(s->n, K, g.t, TB);
    ApplyArgs<R, K> a;
    for (int i = 0; i < (1 << (2 * K)); ++i) {
        a.u[2 * i] = static_cast<R>(g.u[i].real());
        a.u[2 * i + 1] = static_cast<R>(g.u[i].imag());
    }
    a.psi = s->buf;
    a.err = reinterpret_cast<int *>(s->ws + svi::WS_ERR);
    a.ntiles = p.ntiles;
    a.L = p.L;
    a.h = p.h;
    for (int j = 0; j < SV_MAX_K; ++j) a.hi[j] = p.hi[j];
    for (int j = 0; j < K; ++j) a.lp[j] = p.lp[j];
    const unsigned long long cap = (unsigned long long)blocks_per_sm * (unsigned long long)s->num_sms;
    const unsigned grid = (unsigned)std::min<unsigned long long>(p.ntiles, cap);
    const size_t bytes = size_t(1) << (p.L + p.h);
    apply_tile<R, K><<<grid, 256, bytes * sizeof(C), s->stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

}  // namespace svk

namespace svi {

sv_status launch_apply(sv_state *s, const Gate &g, uint64_t *bytes, int *kind) {
    if (g.k < 1 || g.k > SV_MAX_K || g.k > s->n)
        return set_error(SV_ERR_ARG, "apply: gate width out of range");
    if (!(s->policy & SV_POLICY_DENSE_ONLY)) {
        const Structure st = classify(g);
        if (struct_preferred(s, st)) {
            if (kind) *kind = PASS_STRUCTURED;
            return launch_apply_struct(s, st, bytes);
        }
    }
    if (bytes) *bytes = 2ull * ((s->dtype == SV_C64 ? 8ull : 16ull) << s->n);
    if (kind) *kind = PASS_TENSOR_CORE;
    if (tc_eligible(s, g)) return launch_apply_tc(s, g);
    if (tc64_eligible(s, g)) return launch_apply_tc64(s, g);
    if (kind) *kind = PASS_CUDA_CORE;
    if (s->dtype == SV_C64) {
        switch (g.k) {
            case 1: return svk::launch_apply_t<float, 1>(s, g);
            case 2: return svk::launch_apply_t<float, 2>(s, g);
            case 3: return svk::launch_apply_t<float, 3>(s, g);
            case 4: return svk::launch_apply_t<float, 4>(s, g);
            default: return svk::launch_apply_t<float, 5>(s, g);
        }
    }
    switch (g.k) {
        case 1: return svk::launch_apply_t<double, 1>(s, g);
        case 2: return svk::launch_apply_t<double, 2>(s, g);
        case 3: return svk::launch_apply_t<double, 3>(s, g);
        case 4: return svk::launch_apply_t<double, 4>(s, g);
        default: return svk::launch_apply_t<double, 5>(s, g);
    }
}

}  // namespace svi
