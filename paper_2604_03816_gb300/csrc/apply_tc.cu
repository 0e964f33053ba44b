// Fused k = 4, 5 gates in complex64 on the 5th-generation tensor cores (tcgen05).
//
// Per group of 2^k amplitudes the update v' = U v (Eq. 3 with k targets) is a real
// dense contraction: with amplitudes interleaved (re, im), v' = R v where R is the
// 2^{k+1} x 2^{k+1} real embedding of U
//     R[2j][2l] = Re U[j][l],  R[2j][2l+1] = -Im U[j][l],
//     R[2j+1][2l] = Im U[j][l], R[2j+1][2l+1] = Re U[j][l].
// A tile of 128 groups is therefore the GEMM D[128 x N] = A[128 x K] B[N x K]^T with
// A = the groups' amplitudes, B = R and N = K = 2^{k+1} (64 for k = 5, 32 for k = 4).
// TF32 keeps 10 mantissa bits, too few for the complex64 accuracy target, so each
// operand is split into TF32 parts x = x_hi + x_lo (both rounded to nearest) and
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in tensor memory
// (the A_lo B_lo term, of relative size 2^-22, is dropped).
//
// Data flow of one CTA (128 threads, one group per thread, persistent over tiles):
//   TMA 1-D bulk loads of the tile's 2^h segments into a ring of NS raw stages ->
//   each thread gathers its group from the raw stage, splits it and writes row g of
//   A_hi / A_lo in the K-major canonical layout -> one thread issues the 3 x K/8 MMAs
//   into TMEM and commits them to an mbarrier -> each thread reads its row of D with
//   tcgen05.ld and scatters the outputs back into a staging tile -> TMA bulk stores.
// Loads of the next NS tiles are in flight while a tile is processed; the store of a
// tile overlaps the next tile's gather.  All waits are bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "plan.h"
#include "ptx.cuh"
#include "sv_internal.h"
#include "tc.cuh"

namespace svk {

template <int K>
struct TcArgs {
    // U split into TF32 parts on the host from the FP64 matrix, row-major.
    float uhr[1 << (2 * K)], uhi[1 << (2 * K)], ulr[1 << (2 * K)], uli[1 << (2 * K)];
    void *psi;
    int *err;
    unsigned long long ntiles;
    uint32_t L, h;
    uint32_t hi[SV_MAX_K];
    uint32_t lp[K];
};

template <int K>
struct TcShape {
    static constexpr uint32_t D = 1u << K;            // amplitudes per group
    static constexpr uint32_t KD = 2u * D;            // real K = N
    static constexpr uint32_t ROWS = 128;             // groups per tile (MMA M)
    static constexpr uint32_t TB = K + 7;             // tile bits
    static constexpr uint32_t TILE_BYTES = ROWS * D * 8u;
    static constexpr uint32_t A_BYTES = ROWS * KD * 4u;   // == TILE_BYTES
    static constexpr uint32_t B_BYTES = KD * KD * 4u;
    static constexpr uint32_t SBO = (KD / 4u) * 128u;     // 8-row group stride
    static constexpr uint32_t NS = K == 5 ? 3u : 4u;      // raw stages
    static constexpr uint32_t SMEM = 2u * B_BYTES + 2u * A_BYTES + NS * TILE_BYTES;
};

template <int K>
__global__ void __launch_bounds__(128, 1) apply_tc(const __grid_constant__ TcArgs<K> a) {
    using S = TcShape<K>;
    constexpr uint32_t D = S::D, KD = S::KD, NS = S::NS;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long full[NS];
    __shared__ __align__(8) unsigned long long mma_bar;
    __shared__ uint32_t tmem_slot;
    // B first, so that operand reads stay inside the CTA's shared memory whatever the
    // descriptor strides.
    unsigned char *sBh = smem, *sBl = smem + S::B_BYTES;
    unsigned char *sAh = smem + 2 * S::B_BYTES, *sAl = sAh + S::A_BYTES;
    float2 *raw0 = reinterpret_cast<float2 *>(sAl + S::A_BYTES);
    float2 *stage_out = reinterpret_cast<float2 *>(sAh);   // outputs reuse A_hi
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    const uint32_t tid = threadIdx.x, warp = tid >> 5;

    const uint32_t seg_amps = 1u << a.L;
    const uint32_t seg_bytes = seg_amps * 8u;
    const uint32_t nseg = 1u << a.h;

    // ---- set-up: TMEM, barriers, B = R split into TF32 parts
    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_slot), KD);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (uint32_t s = 0; s < NS; ++s) mbar_init(smem_u32(&full[s]), 1);
        mbar_init(smem_u32(&mma_bar), 1);
        fence_mbar_init();
    }
    for (uint32_t e = tid; e < KD * KD; e += blockDim.x) {
        const uint32_t n = e / KD, kk = e % KD;
        const uint32_t j = n >> 1, l = kk >> 1, u = j * D + l;
        float vh, vl;
        if ((n & 1) == (kk & 1)) {                  // Re U on the diagonal of the 2x2 block
            vh = a.uhr[u]; vl = a.ulr[u];
        } else if (n & 1) {                         // R[2j+1][2l] = Im U
            vh = a.uhi[u]; vl = a.uli[u];
        } else {                                    // R[2j][2l+1] = -Im U
            vh = -a.uhi[u]; vl = -a.uli[u];
        }
        const uint32_t off = kmajor_off(n, kk, S::SBO);
        *reinterpret_cast<float *>(sBh + off) = vh;
        *reinterpret_cast<float *>(sBl + off) = vl;
    }
    uint32_t coff[D];
#pragma unroll
    for (uint32_t c = 0; c < D; ++c) {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((c >> j) & 1) o |= 1u << a.lp[j];
        coff[c] = o;
    }
    uint32_t gbase = tid;                           // this thread's group base in the tile
#pragma unroll
    for (int j = 0; j < K; ++j) gbase = insert_zero32(gbase, a.lp[j]);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_tf32(S::ROWS, KD);

    auto tile_base = [&](unsigned long long t) {
        unsigned long long base = t << a.L;
        for (uint32_t j = 0; j < a.h; ++j) base = insert_zero64(base, a.hi[j]);
        return base;
    };
    auto issue_load = [&](unsigned long long t, uint32_t s) {
        const unsigned long long base = tile_base(t);
        const uint32_t bar = smem_u32(&full[s]);
        mbar_arrive_expect_tx(bar, S::TILE_BYTES);
        float2 *dst = raw0 + (size_t)s * (S::TILE_BYTES / 8u);
        for (uint32_t sg = 0; sg < nseg; ++sg) {
            unsigned long long off = base;
            for (uint32_t j = 0; j < a.h; ++j)
                if ((sg >> j) & 1u) off |= 1ull << a.hi[j];
            bulk_g2s(smem_u32(dst + (size_t)sg * seg_amps), psi + off, seg_bytes, bar);
        }
    };

    const unsigned long long first = blockIdx.x, step = gridDim.x;
    if (tid == 0)
        for (uint32_t s = 0; s < NS; ++s) {
            const unsigned long long t = first + s * step;
            if (t < a.ntiles) issue_load(t, s);
        }

    bool failed = false;
    uint32_t it = 0;
    for (unsigned long long t = first; t < a.ntiles; t += step, ++it) {
        const uint32_t s = it % NS;
        const uint32_t par = (it / NS) & 1u;
        if (tid == 0) bulk_wait_read_all();          // previous tile's store left A_hi
        const bool ok = mbar_wait_bounded(smem_u32(&full[s]), par);
        if (!__syncthreads_and(ok)) { failed = true; break; }

        // gather this thread's group, split into TF32 parts, write row `tid` of A
        const float2 *rs = raw0 + (size_t)s * (S::TILE_BYTES / 8u);
#pragma unroll 8
        for (uint32_t c = 0; c < D; ++c) {
            const float2 v = rs[gbase | coff[c]];
            const float hr = tf32_rna(v.x), hi = tf32_rna(v.y);
            const float lr = tf32_rna(v.x - hr), li = tf32_rna(v.y - hi);
            const uint32_t off = kmajor_off(tid, 2 * c, S::SBO);
            *reinterpret_cast<float2 *>(sAh + off) = make_float2(hr, hi);
            *reinterpret_cast<float2 *>(sAl + off) = make_float2(lr, li);
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (tid == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl);
            const uint32_t bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
            for (uint32_t p = 0; p < 3; ++p) {
                const uint32_t A = p == 2 ? al : ah, B = p == 1 ? bl : bh;
#pragma unroll
                for (uint32_t ks = 0; ks < KD / 8; ++ks)
                    mma_tf32(tmem, smem_desc(A + ks * 256u, 128u, S::SBO),
                             smem_desc(B + ks * 256u, 128u, S::SBO), idesc, (p | ks) != 0);
            }
            mma_commit(smem_u32(&mma_bar));
            const unsigned long long nt = t + NS * step;   // raw stage s is free again
            if (nt < a.ntiles) issue_load(nt, s);
        }
        const bool ok2 = mbar_wait_bounded(smem_u32(&mma_bar), it & 1u);
        if (!__syncthreads_and(ok2)) { failed = true; break; }
        tc_fence_after();

        // row `tid` of D: outputs of this thread's group, scattered into the staging tile
        float d[KD];
#pragma unroll
        for (uint32_t c0 = 0; c0 < KD; c0 += 32) {
            float part[32];
            tmem_ld32(tmem + ((warp * 32u) << 16) + c0, part);
#pragma unroll
            for (int i = 0; i < 32; ++i) d[c0 + i] = part[i];
        }
        tmem_wait_ld();
#pragma unroll
        for (uint32_t c = 0; c < D; ++c) stage_out[gbase | coff[c]] = make_float2(d[2 * c], d[2 * c + 1]);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            const unsigned long long base = tile_base(t);
            for (uint32_t sg = 0; sg < nseg; ++sg) {
                unsigned long long off = base;
                for (uint32_t j = 0; j < a.h; ++j)
                    if ((sg >> j) & 1u) off |= 1ull << a.hi[j];
                bulk_s2g(psi + off, smem_u32(stage_out + (size_t)sg * seg_amps), seg_bytes);
            }
            bulk_commit();
        }
    }
    if (failed && tid == 0) atomicOr(a.err, 2);
    if (tid == 0) bulk_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, KD);
}

// Host: round to TF32 (10 mantissa bits), nearest with ties away from zero, like
// cvt.rna.tf32.f32.
static float tf32_host(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0x7F800000u) != 0x7F800000u) {
        b += 0x1000u;
        b &= ~0x1FFFu;
    }
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

template <int K>
sv_status launch_tc_t(sv_state *s, const svi::Gate &g) {
    using S = TcShape<K>;
    static std::once_flag once;
    static cudaError_t init_err = cudaSuccess;
    std::call_once(once, [] {
        init_err = cudaFuncSetAttribute(apply_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)S::SMEM);
    });
    if (init_err != cudaSuccess)
        return svi::set_error(SV_ERR_CUDA, std::string("tensor-core kernel setup: ") +
                                               cudaGetErrorString(init_err));
    const Plan p = make_plan(s->n, K, g.t, S::TB);
    TcArgs<K> a;
    for (int i = 0; i < (1 << (2 * K)); ++i) {
        const double re = g.u[i].real(), im = g.u[i].imag();
        a.uhr[i] = tf32_host((float)re);
        a.uhi[i] = tf32_host((float)im);
        a.ulr[i] = tf32_host((float)(re - (double)a.uhr[i]));
        a.uli[i] = tf32_host((float)(im - (double)a.uhi[i]));
    }
    a.psi = s->buf;
    a.err = reinterpret_cast<int *>(s->ws + svi::WS_ERR);
    a.ntiles = p.ntiles;
    a.L = p.L;
    a.h = p.h;
    for (int j = 0; j < SV_MAX_K; ++j) a.hi[j] = p.hi[j];
    for (int j = 0; j < K; ++j) a.lp[j] = p.lp[j];
    const int per_sm = (int)std::max<uint32_t>(1u, (227u * 1024u) / (S::SMEM + 2048u));
    const unsigned grid = (unsigned)std::min<unsigned long long>(p.ntiles,
                                                                 (unsigned long long)per_sm * s->num_sms);
    apply_tc<K><<<grid, 128, S::SMEM, s->stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

}  // namespace svk

namespace svi {

bool tc_eligible(const sv_state *s, const Gate &g) {
    return s->dtype == SV_C64 && (g.k == 4 || g.k == 5) && s->n >= g.k + 7 &&
           !(s->policy & SV_POLICY_NO_TENSOR_CORES);
}

sv_status launch_apply_tc(sv_state *s, const Gate &g) {
    return g.k == 5 ? svk::launch_tc_t<5>(s, g) : svk::launch_tc_t<4>(s, g);
}

}  // namespace svi
