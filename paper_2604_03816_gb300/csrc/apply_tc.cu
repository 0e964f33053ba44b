// Fused k = 4, 5 gates in complex64 on the 5th-generation tensor cores (tcgen05).
//
// Per group of 2^k amplitudes the update v' = U v (Eq. 3 with k targets) is a real
// dense contraction: with amplitudes interleaved (re, im), v' = R v where R is the
// 2^{k+1} x 2^{k+1} real embedding of U
//     R[2j][2l] = Re U[j][l],  R[2j][2l+1] = -Im U[j][l],
//     R[2j+1][2l] = Im U[j][l], R[2j+1][2l+1] = Re U[j][l].
// A tile of 128 groups is the GEMM D[128 x N] = A[128 x K] B[N x K]^T with A = the
// groups' amplitudes, B = R and N = K = 2^{k+1} (64 for k = 5, 32 for k = 4).
//
// Precision: the tensor cores' FP32 accumulation truncates, so a plain split of the
// FP32 operands into TF32 parts gives errors biased toward zero (a measurable loss of
// norm per pass).  Instead each operand is cut into three 9-bit integer slices on a
// fixed-point grid -- per row of A (scale 2^{8-e}, e = exponent of the row's largest
// component) and for all of B -- so that x = (a1 + a2 2^-9 + a3 2^-18) / s.  The
// slices are exact in FP16 and every product of integer slices is below 2^16, so
//     D0  = A1 B1                                      (below 2^22: exact in FP32)
//     D12 = A1 B2 + A2 B1 + 2^-9 (A1 B3 + A2 B2 + A3 B1)
// are accumulated by the tensor cores (kind::f16, FP32 accumulators in TMEM); the
// 2^-9-scaled slices (B3, B2 and A3 times 2^-9) are also exact in FP16.  D0, which
// carries the leading 2^22 of the result, is exact; D12 sits 2^-9 below it, so the
// truncation of its accumulation costs about 2^-31 of the output per step -- the error
// stays unbiased to well below FP32 rounding.  The epilogue forms
// out = (D0 + 2^-9 D12) / (s s_B) with round-to-nearest (the dropped slice products are
// below 2^-27 of the row's largest amplitude).
//
// One persistent CTA per SM, warp-specialised, every hand-off an mbarrier:
//   warp 8               TMA producer: lane i issues the load of segment i of each tile
//                        into a ring of NS raw stages (a 1-D bulk copy, or 2-D tensor-map
//                        boxes of 128-byte rows with the 128-byte swizzle, SW);
//   warps 0-7            transform: two warps per TMEM lane quadrant, one group (row of A)
//                        and half of its members per thread -- gather from the raw stage,
//                        cut into three 9-bit slices and write them into tensor memory
//                        with tcgen05.st (the thread's own TMEM lane);
//   warp 9 (one thread)  MMA issuer: 6 x K/16 tcgen05.mma.kind::f16, A from TMEM and B
//                        from shared memory, into two TMEM accumulators
//                        (double-buffered), committed to mbarriers;
//   warps 10-17          epilogue: two warps per quadrant, tcgen05.ld of half the columns,
//                        combine, scatter into an output staging tile; warp 10 issues the
//                        TMA bulk stores.
// Targets among tile bits 0..3 (where 8-byte accesses pick their bank) would make the
// lanes of a warp hit one bank.  Width-5 launches on states of 13 qubits or more, and
// batched launches, avoid that with the swizzled staging (SW); the others (11- and
// 12-qubit states) take each group's members in a lane-dependent XOR order (XP), undone
// in registers.
// So loads, slicing, MMAs and stores of consecutive tiles overlap.  With A in tensor
// memory, shared memory holds only B, the raw stages and the output staging, so 4 (k = 5)
// or 8 (k = 4) tiles of loads can be in flight per SM.  Every wait is bounded and any
// role that gives up makes the others leave too (abort flag).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "plan.h"
#include "ptx.cuh"
#include "sv_internal.h"
#include "tc.cuh"

namespace svk {

// SUB: MMA subtiles (128 groups each) per TMA stage.  SUB = 2 doubles the contiguous
// segments of launches whose targets are all high (2 KiB instead of 1 KiB at k = 5), at
// the price of one more A slice in TMEM (A2 2^-9 replaces the B2 2^-9 copy, to fit two
// 64 KiB stages in shared memory).
// BT: a batched launch over many states with their own matrices (see apply_tc): two B
// sets (the current state's and the next one's) and two raw stages.
template <int K, int SUB = 1, bool BT = false>
struct TcShape {
    static constexpr uint32_t D = 1u << K;            // amplitudes per group
    static constexpr uint32_t KD = 2u * D;            // real K = N
    static constexpr uint32_t ROWS = 128;             // groups per MMA subtile (MMA M)
    static constexpr uint32_t TB = K + 7 + (SUB == 2 ? 1u : 0u);   // tile bits
    static constexpr uint32_t TILE_BYTES = SUB * ROWS * D * 8u;
    static constexpr uint32_t B_BYTES = KD * KD * 2u;     // one FP16 slice of B
    static constexpr uint32_t NB = SUB == 2 ? 3u : 4u;    // B1, B2, B3 2^-9 [, B2 2^-9]
    static constexpr uint32_t SBO = (KD / 8u) * 128u;     // 8-row group stride of B
    static constexpr uint32_t NS = (SUB == 2 || BT) ? 2u : (K == 5 ? 3u : 8u);   // raw stages
    static constexpr uint32_t NOUT = SUB == 2 ? 1u : 2u;  // output staging tiles
    static constexpr uint32_t ACC = 2u * KD;              // TMEM columns of one D set (D0, D12)
    static constexpr uint32_t A_COLS = KD / 2u;           // TMEM columns of one A slice
    static constexpr uint32_t NA = SUB == 2 ? 4u : 3u;    // A1, A2, A3 2^-9 [, A2 2^-9]
    static constexpr uint32_t A_SET = NA * A_COLS;        // one A buffer
    static constexpr uint32_t A_COL0 = 2u * ACC;          // first column of the A buffers
    static constexpr uint32_t TMEM_COLS = K == 5 ? 512u : 256u;
    static_assert(A_COL0 + 2u * A_SET <= TMEM_COLS, "TMEM layout");
    static constexpr uint32_t NBSET = BT ? 2u : 1u;       // B sets
    static constexpr uint32_t B_SET = NB * B_BYTES;
    static constexpr uint32_t OFF_RAW = NBSET * B_SET;
    static constexpr uint32_t OFF_OUT = OFF_RAW + NS * TILE_BYTES;
    static constexpr uint32_t SMEM = OFF_OUT + NOUT * TILE_BYTES;
    static constexpr uint32_t THREADS = 576;              // 18 warps
    // warps 0-7 transform, 8 TMA producer, 9 MMA issuer, 10-17 epilogue
    static constexpr uint32_t W_PROD = 8, W_MMA = 9, W_EPI = 10;
    static constexpr uint32_t HALF = D / 2;               // group members per worker thread
};

template <int K>
struct TcArgs {
    // swizzled launches (SW): the state as a 2-D tensor of 128-byte rows (32 floats), boxes
    // of box_rows rows, `boxes` boxes per segment, 128-byte swizzle in shared memory
    CUtensorMap tmap;                      // 128-byte aligned by its type
    uint32_t box_rows, boxes;
    int16_t b[3][(2u << K) * (2u << K)];   // slices of R (row-major n x kk), |b| <= 256
    float b_inv_scale;                     // R = (b1 + b2 2^-9 + b3 2^-18) * b_inv_scale
    void *psi;
    int *err;
    unsigned long long ntiles;
    uint32_t L, h;
    uint32_t hi[SV_MAX_K];
    uint32_t lp[K];
    // bank-conflict avoidance: the xt lowest targets sit at tile bits below 4; lane l
    // takes group members in the order c ^ x(l), x(l) = (l >> xs) & (2^xt - 1)
    uint32_t xs, xt;
    // batched launches: ntiles = states x tiles_per_state, state i at amplitude offset
    // i 2^n; state i's matrix is utab + i 2 4^kin (FP32 complex, row-major), of width kin
    // = K, or K - 1 widened by an identity qubit at local bit jw (jw = -1: not widened)
    const float *utab;
    unsigned long long tiles_per_state;
    uint32_t n, kin;
    int jw;
};

// v[c] <- v[c ^ x] for the low xt bits of x: one conditional-swap stage per bit.
template <int N>
__device__ __forceinline__ void xor_unpermute(float2 (&v)[N], uint32_t x, uint32_t xt) {
    constexpr int NBITS = N >= 16 ? 4 : (N >= 8 ? 3 : (N >= 4 ? 2 : 1));
#pragma unroll
    for (int j = 0; j < NBITS; ++j) {
        if (xt > (uint32_t)j) {                       // uniform over the launch
            const bool f = (x >> j) & 1u;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                if (c & (1 << j)) continue;
                const float2 lo = v[c], hi = v[c | (1 << j)];
                v[c] = make_float2(f ? hi.x : lo.x, f ? hi.y : lo.y);
                v[c | (1 << j)] = make_float2(f ? lo.x : hi.x, f ? lo.y : hi.y);
            }
        }
    }
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);   // exact: |a|, |b| <= 256 are integers
    return *reinterpret_cast<const uint32_t *>(&h);
}

// An FP16 pair times 2^-9 (exact for the integer slices: at most 9 bits, no underflow).
__device__ __forceinline__ uint32_t half2_times_2m9(uint32_t w) {
    const __half2 h = __hmul2(*reinterpret_cast<const __half2 *>(&w), __float2half2_rn(1.f / 512.f));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Three 9-bit integer slices of a scaled amplitude (|x scale| < 256): FP16 pairs
// (re, im) of a1, a2 and a3 2^-9, all exact.
__device__ __forceinline__ void slice3(float2 v, float scale, uint32_t &w1, uint32_t &w2, uint32_t &w3) {
    const float xr = v.x * scale, xi = v.y * scale;
    const float r1 = rintf(xr), i1 = rintf(xi);
    const float xr2 = (xr - r1) * 512.f, xi2 = (xi - i1) * 512.f;
    const float r2 = rintf(xr2), i2 = rintf(xi2);
    const float r3 = rintf((xr2 - r2) * 512.f), i3 = rintf((xi2 - i2) * 512.f);
    w1 = pack_half2(r1, i1);
    w2 = pack_half2(r2, i2);
    w3 = pack_half2(r3 * (1.f / 512.f), i3 * (1.f / 512.f));
}

// Batched launches build B in shared memory from a state's FP32 matrix (width kin, or
// K - 1 widened by an identity qubit at local bit jw): entry (r, c) of the K-qubit U.
__device__ __forceinline__ float u_entry(const float *U, uint32_t kin, int jw, uint32_t r, uint32_t c,
                                         uint32_t part) {
    if (jw >= 0) {
        if (((r ^ c) >> jw) & 1u) return 0.f;
        const uint32_t lo = (1u << jw) - 1u;
        r = (r & lo) | ((r >> (jw + 1)) << jw);
        c = (c & lo) | ((c >> (jw + 1)) << jw);
    }
    return U[2u * ((r << kin) + c) + part];
}

// Largest |entry| of a state's stored matrix over the entries i0, i0 + stride, ...
__device__ __forceinline__ float u_absmax_part(const float *U, uint32_t kin, uint32_t i0, uint32_t stride) {
    float m = 0.f;
    for (uint32_t i = i0; i < (2u << (2u * kin)); i += stride) m = fmaxf(m, fabsf(U[i]));
    return m;
}

// B = the four FP16 slices (B1, B2, B3 2^-9, B2 2^-9) of R x sb, R the real embedding of
// the state's U and sb = 2^(8 - eb) with max |R| < 2^eb, so |R sb| < 256 and the three
// 9-bit slices of the FP32 value are exact; entries i0, i0 + stride, ...
template <int K>
__device__ void build_b(unsigned char *sB, const float *U, uint32_t kin, int jw, float sb, uint32_t i0,
                        uint32_t stride) {
    using S = TcShape<K, 1, true>;
    constexpr uint32_t KD = S::KD;
    for (uint32_t e = i0; e < KD * KD; e += stride) {
        const uint32_t n = e / KD, kk = e % KD, r = n >> 1, c = kk >> 1;
        float v;
        if ((n & 1u) == (kk & 1u)) v = u_entry(U, kin, jw, r, c, 0);
        else v = (n & 1u) ? u_entry(U, kin, jw, r, c, 1) : -u_entry(U, kin, jw, r, c, 1);
        const float x = v * sb;
        const float b1 = rintf(x);
        const float x2 = (x - b1) * 512.f;
        const float b2 = rintf(x2);
        const float b3 = rintf((x2 - b2) * 512.f);
        const uint32_t off = kmajor_off16(n, kk, S::SBO);
        *reinterpret_cast<__half *>(sB + 0 * S::B_BYTES + off) = __float2half_rn(b1);
        *reinterpret_cast<__half *>(sB + 1 * S::B_BYTES + off) = __float2half_rn(b2);
        *reinterpret_cast<__half *>(sB + 2 * S::B_BYTES + off) = __float2half_rn(b3 * (1.f / 512.f));
        *reinterpret_cast<__half *>(sB + 3 * S::B_BYTES + off) = __float2half_rn(b2 * (1.f / 512.f));
    }
}

// sb = 2^(8 - eb) and 1 / sb for a matrix whose largest |entry| is m < 2^eb.
__device__ __forceinline__ void b_grid(float m, float &sb, float &inv) {
    int eb = 0;
    frexpf(m, &eb);
    eb = max(eb, -100);
    sb = ldexpf(1.f, 8 - eb);
    inv = ldexpf(1.f, eb - 8);
}

// XP: the launch has targets among tile bits 0..3 and takes members in the lane's XOR
// order; otherwise every lane takes them in member order (no permutation code at all).
// The pipelines count tiles (j: raw stage, output staging) and MMA subtiles (js = j SUB +
// sub: A and D buffers, row scales).
// BT: one launch over a batch of states, each with its own matrix: a CTA takes a
// contiguous range of tiles (so it meets few states), B is double-buffered and rebuilt by
// the producer warp from the next state's matrix when its first tile comes up (b_full:
// built; b_empty: the MMAs of the state that last used the set have completed).
// SW: tiles move by 2-D tensor-map copies that store them in shared memory with the
// 128-byte swizzle (16-byte chunk index XOR the 128-byte row within each 1 KiB), and the
// roles address the tile through the same swizzle.  A warp's lanes (consecutive groups)
// then reach different banks whatever the targets, so no lane-dependent member order is
// needed (XP = false) and every layout takes two subtiles per stage.  The swizzle is linear
// over XOR, so it is applied to the group base and to the target bits once, and member
// offsets combine them by XOR.
template <int K, bool XP, int SUB, bool BT = false, bool SW = false>
__global__ void __launch_bounds__(576, 1) apply_tc(const __grid_constant__ TcArgs<K> a) {
    using S = TcShape<K, SUB, BT>;
    constexpr uint32_t KD = S::KD, NS = S::NS, NOUT = S::NOUT, HALF = S::HALF;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long full[NS], empty[NS];
    __shared__ __align__(8) unsigned long long a_full[2], a_empty[2], d_full[2], d_empty[2];
    __shared__ __align__(8) unsigned long long scale_full[4];   // row scales, tile j -> j & 3
    __shared__ float row_scale[4][128];
    __shared__ float max_part[2][128];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ __align__(8) unsigned long long b_full[2], b_empty[2];   // batched launches
    __shared__ float b_scale[2];
    __shared__ float red[32];
    // B slices, the raw stages and the output staging tiles; B operand reads stay inside
    // the CTA's shared memory whatever the descriptor strides.
    unsigned char *sB = smem;
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const uint32_t seg_amps = 1u << a.L;
    const uint32_t seg_bytes = seg_amps * 8u;
    const uint32_t nseg = 1u << a.h;

    if (warp == S::W_MMA) {
        tmem_alloc(smem_u32(&tmem_slot), S::TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (uint32_t s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&a_full[b]), 1);
            mbar_init(smem_u32(&a_empty[b]), 1);
            mbar_init(smem_u32(&d_full[b]), 1);
            mbar_init(smem_u32(&d_empty[b]), 1);
        }
        for (int q = 0; q < 4; ++q) mbar_init(smem_u32(&scale_full[q]), 1);
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&b_full[q]), 1);
            mbar_init(smem_u32(&b_empty[q]), 1);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    // tiles of this CTA: strided over the grid, or (batched) a contiguous range
    unsigned long long first = blockIdx.x, step = gridDim.x, tend = a.ntiles;
    if constexpr (BT) {
        const unsigned long long per = (a.ntiles + gridDim.x - 1) / gridDim.x;
        first = min(a.ntiles, (unsigned long long)blockIdx.x * per);
        tend = min(a.ntiles, first + per);
        step = 1;
    }
    if constexpr (BT) {
        // B set 0 from the matrix of the range's first state, built by every thread
        const unsigned long long st0 = first < tend ? first / a.tiles_per_state : 0;
        const float *U0 = a.utab + st0 * (2ull << (2u * a.kin));
        float m = u_absmax_part(U0, a.kin, tid, blockDim.x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red[warp] = m;
        __syncthreads();
        m = 0.f;
        for (uint32_t w = 0; w < S::THREADS / 32u; ++w) m = fmaxf(m, red[w]);
        float sb, inv;
        b_grid(m, sb, inv);
        build_b<K>(sB, U0, a.kin, a.jw, sb, tid, blockDim.x);
        if (tid == 0) b_scale[0] = inv;
    } else {
        for (uint32_t e = tid; e < KD * KD; e += blockDim.x) {
            const uint32_t n = e / KD, kk = e % KD, off = kmajor_off16(n, kk, S::SBO);
            *reinterpret_cast<__half *>(sB + 0 * S::B_BYTES + off) = __int2half_rn(a.b[0][e]);
            *reinterpret_cast<__half *>(sB + 1 * S::B_BYTES + off) = __int2half_rn(a.b[1][e]);
            // exact: integers below 2^9 times 2^-9
            *reinterpret_cast<__half *>(sB + 2 * S::B_BYTES + off) = __float2half_rn(a.b[2][e] * (1.f / 512.f));
            if constexpr (SUB == 1)
                *reinterpret_cast<__half *>(sB + 3 * S::B_BYTES + off) = __float2half_rn(a.b[1][e] * (1.f / 512.f));
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if constexpr (BT) {
        if (tid == 0) mbar_arrive(smem_u32(&b_full[0]));   // set 0: its first use
    }
    const uint32_t tmem = tmem_slot;
    volatile int *abort = &abort_flag;
    // amplitude offset of tile t (batched: the state's offset plus the tile's base)
    auto tile_base = [&](const SegLanes &sl, unsigned long long t) -> unsigned long long {
        if constexpr (BT) {
            const unsigned long long st = t / a.tiles_per_state;
            return (st << a.n) + sl.base(t - st * a.tiles_per_state);
        } else {
            return sl.base(t);
        }
    };

    auto group_base = [&](uint32_t row) {
        uint32_t g = row;
#pragma unroll
        for (int j = 0; j < K; ++j) g = insert_zero32(g, a.lp[j]);
        return SW ? swz128(g) : g;
    };
    // offset of group member c (bit j of c at tile bit lp[j]); for the unrolled constant
    // c this is an XOR of the (swizzled) bits 1 << lp[j] held in K registers, and a
    // member's index is group base XOR offset
    uint32_t tbit[K];
#pragma unroll
    for (int j = 0; j < K; ++j) tbit[j] = SW ? swz128(1u << a.lp[j]) : 1u << a.lp[j];
    auto member_off = [&](uint32_t c) {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((c >> j) & 1u) o ^= tbit[j];
        return o;
    };

    if (warp == S::W_PROD) {
        // ------------------------------------------------------------ TMA producer
        // lane i issues the bulk copy of segment i of every tile
        SegLanes sl;
        sl.init(a.L, a.h, a.hi, lane);
        uint32_t j = 0;
        unsigned long long cur = ~0ull;
        uint32_t nsw = 0;                         // state changes so far (B set = nsw & 1)
        for (unsigned long long t = first; t < tend; t += step, ++j) {
            if constexpr (BT) {
                const unsigned long long st = t / a.tiles_per_state;
                if (cur == ~0ull) {
                    cur = st;                     // set 0 was built at the start
                } else if (st != cur) {
                    cur = st;
                    ++nsw;
                    const uint32_t set = nsw & 1u, use = nsw >> 1;
                    bool okb = true;
                    if (use >= 1 && lane == 0)
                        okb = mbar_wait_or_abort(smem_u32(&b_empty[set]), (use - 1u) & 1u, abort);
                    if (!__shfl_sync(0xffffffffu, (int)okb, 0)) break;
                    const float *U = a.utab + st * (2ull << (2u * a.kin));
                    float m = u_absmax_part(U, a.kin, lane, 32);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                    float sb, inv;
                    b_grid(m, sb, inv);
                    build_b<K>(sB + set * S::B_SET, U, a.kin, a.jw, sb, lane, 32);
                    if (lane == 0) b_scale[set] = inv;
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&b_full[set]));
                }
            }
            const uint32_t s = j % NS, u = j / NS;
            bool ok = true;
            if (lane == 0) ok = mbar_wait_or_abort(smem_u32(&empty[s]), (u & 1u) ^ 1u, abort);
            if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
            const uint32_t bar = smem_u32(&full[s]);
            if (lane == 0) mbar_arrive_expect_tx(bar, S::TILE_BYTES);
            __syncwarp();
            if (lane < nseg) {
                float2 *dst = reinterpret_cast<float2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
                if constexpr (SW) {
                    // segment = `boxes` boxes of box_rows 128-byte rows (16 amplitudes each)
                    const int32_t row0 = (int32_t)((tile_base(sl, t) + sl.my_off) >> 4);
                    const uint32_t d0 = smem_u32(dst + (size_t)lane * seg_amps);
                    for (uint32_t bx = 0; bx < a.boxes; ++bx)
                        tma_load_2d(d0 + bx * a.box_rows * 128u, &a.tmap, 0, row0 + (int32_t)(bx * a.box_rows), bar);
                } else {
                    bulk_g2s(smem_u32(dst + (size_t)lane * seg_amps), psi + tile_base(sl, t) + sl.my_off,
                             seg_bytes, bar);
                }
            }
        }
    } else if (warp == S::W_MMA) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(S::ROWS, KD);
            uint32_t B0 = smem_u32(sB);
            const unsigned long long nsub = tend > first ? ((tend - first + step - 1) / step) * SUB : 0;
            unsigned long long cur = ~0ull;
            uint32_t nsw = 0;
            for (unsigned long long js = 0; js < nsub; ++js) {
                if constexpr (BT) {
                    const unsigned long long st = (first + (js / SUB) * step) / a.tiles_per_state;
                    if (st != cur) {
                        if (cur != ~0ull) {
                            mma_commit(smem_u32(&b_empty[nsw & 1u]));   // the old state's MMAs
                            ++nsw;
                        }
                        cur = st;
                        const uint32_t set = nsw & 1u, use = nsw >> 1;
                        if (!mbar_wait_or_abort(smem_u32(&b_full[set]), use & 1u, abort)) break;
                        tc_fence_after();
                        B0 = smem_u32(sB) + set * S::B_SET;
                    }
                }
                const uint32_t b = (uint32_t)js & 1u, u = (uint32_t)(js >> 1);
                if (!mbar_wait_or_abort(smem_u32(&a_full[b]), u & 1u, abort)) break;
                if (!mbar_wait_or_abort(smem_u32(&d_empty[b]), (u & 1u) ^ 1u, abort)) break;
                tc_fence_after();
                const uint32_t A0 = tmem + S::A_COL0 + b * S::A_SET;
                const uint32_t dset = tmem + b * S::ACC;
                // (accumulator, A slice, B slice): D0 = A1 B1; D12 = A1 B2 + A2 B1 +
                // A1 (B3 2^-9) + A2 (B2 2^-9) + (A3 2^-9) B1   [A slices: A1, A2, A3s, A2s;
                // B slices: B1, B2, B3s, B2s]; with SUB = 2, A2s B2 stands for A2 B2s
                const uint32_t prod[6][3] = {{0, 0, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 2},
                                             {1, SUB == 2 ? 3u : 1u, SUB == 2 ? 1u : 3u}, {1, 2, 0}};
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint32_t Aa = A0 + prod[p][1] * S::A_COLS;
                    const uint32_t Bb = B0 + prod[p][2] * S::B_BYTES;
                    const bool first_in_acc = (p == 0 || p == 1);
#pragma unroll
                    for (uint32_t ks = 0; ks < KD / 16; ++ks)
                        mma_f16_tmem_a(dset + prod[p][0] * KD, Aa + ks * 8u,
                                       smem_desc(Bb + ks * 256u, 128u, S::SBO), idesc,
                                       (first_in_acc && ks == 0) ? 0u : 1u);
                }
                mma_commit(smem_u32(&a_empty[b]));
                mma_commit(smem_u32(&d_full[b]));
            }
        }
    } else if (warp < S::W_PROD) {
        // ------------------------------------------------------------ transform
        // Two warps per TMEM lane quadrant: warp w takes rows 32 (w & 3) .. + 31 of each MMA
        // subtile and group members HALF (w >> 2) .. + HALF - 1.
        const uint32_t row = (warp & 3u) * 32u + lane;
        const uint32_t part = warp >> 2;
        uint32_t gb[SUB];
#pragma unroll
        for (uint32_t sub = 0; sub < SUB; ++sub) gb[sub] = group_base(sub * S::ROWS + row);
        const uint32_t xl = (lane >> a.xs) & ((1u << a.xt) - 1u);
        uint32_t cx = 0;
#pragma unroll
        for (int q = 0; q < K; ++q)
            if ((xl >> q) & 1u) cx |= tbit[q];
        uint32_t j = 0;
        bool stop = false;
        unsigned long long cur = ~0ull;
        uint32_t nsw = 0;
        for (unsigned long long t = first; t < tend && !stop; t += step, ++j) {
            if constexpr (BT) {
                const unsigned long long st = t / a.tiles_per_state;
                if (cur != ~0ull && st != cur) ++nsw;
                cur = st;
            }
            const uint32_t s = j % NS;
            const bool okf = mbar_wait_or_abort(smem_u32(&full[s]), (j / NS) & 1u, abort);
            const float2 *rs = reinterpret_cast<const float2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
#pragma unroll
            for (uint32_t sub = 0; sub < SUB; ++sub) {
                const uint32_t js = j * SUB + sub;
                const uint32_t gbase = gb[sub];
                // this half of the row (members in the lane's order c ^ x), its largest component
                float2 v[HALF];
                float m = 0.f;
#pragma unroll
                for (uint32_t c = 0; c < HALF; ++c) {
                    const uint32_t mo = member_off(part * HALF + c);
                    v[c] = rs[gbase ^ (XP ? (mo ^ cx) : mo)];
                    m = fmaxf(m, fmaxf(fabsf(v[c].x), fabsf(v[c].y)));
                }
                max_part[part][row] = m;
                fence_proxy_async_smem();         // reads of the raw stage before its refill
                if (!named_bar_and(1, 256, okf)) { stop = true; break; }
                if (sub == SUB - 1 && tid == 0) mbar_arrive(smem_u32(&empty[s]));
                m = fmaxf(max_part[0][row], max_part[1][row]);
                int ex = 0;
                frexpf(m, &ex);                   // m < 2^ex (m = 0: ex = 0)
                ex = max(ex, -100);               // keep 2^(8-ex) finite
                const float scale = ldexpf(1.f, 8 - ex);   // |x * scale| < 256
                const uint32_t ab = js & 1u;
                const bool oka = mbar_wait_or_abort(smem_u32(&a_empty[ab]), ((js >> 1) & 1u) ^ 1u, abort);
                if (!named_bar_and(1, 256, oka)) { stop = true; break; }
                tc_fence_after();
                // slot js & 3 was last read by the epilogue of subtile js - 4, which finished
                // before the MMAs of subtile js - 2 were issued, whose completion released
                // a_empty[ab]
                // batched: the state's B scale, written by the producer before this tile's load
                if (part == 0) row_scale[js & 3u][row] = ldexpf(BT ? b_scale[nsw & 1u] : a.b_inv_scale, ex - 8);
                if constexpr (XP) xor_unpermute(v, xl, a.xt);   // back in member order (x < HALF)
                // three 9-bit integer slices (and A2 2^-9 when SUB = 2), one FP16 pair
                // (re, im) per 32-bit TMEM column, stored eight members at a time
                const uint32_t arow = tmem + S::A_COL0 + ab * S::A_SET + (((warp & 3u) * 32u) << 16) +
                                      part * HALF;
#pragma unroll
                for (uint32_t c0 = 0; c0 < HALF; c0 += 8) {
                    uint32_t w1[8], w2[8], w3[8], w2s[8];
#pragma unroll
                    for (uint32_t c = 0; c < 8; ++c) {
                        slice3(v[c0 + c], scale, w1[c], w2[c], w3[c]);
                        if constexpr (SUB == 2) w2s[c] = half2_times_2m9(w2[c]);
                    }
                    tmem_st8_async(arow + c0, w1);
                    tmem_st8_async(arow + S::A_COLS + c0, w2);
                    tmem_st8_async(arow + 2 * S::A_COLS + c0, w3);
                    if constexpr (SUB == 2) tmem_st8_async(arow + 3 * S::A_COLS + c0, w2s);
                }
                tmem_wait_st();
                tc_fence_before();
                named_bar(1, 256);                // also: max_part is free for the next subtile
                if (tid == 0) {
                    mbar_arrive(smem_u32(&a_full[ab]));
                    mbar_arrive(smem_u32(&scale_full[js & 3u]));
                }
            }
        }
    } else if (warp >= S::W_EPI) {
        // ------------------------------------------------------------ epilogue
        // Two warps per lane quadrant, each over half of the accumulator columns.
        const uint32_t quad = warp & 3u;          // TMEM lanes 32*quad .. 32*quad+31
        const uint32_t row = quad * 32u + lane;
        const uint32_t et = tid - S::W_EPI * 32u; // 0..255 within the epilogue warps
        const uint32_t part = et >> 7;
        uint32_t gb[SUB];
#pragma unroll
        for (uint32_t sub = 0; sub < SUB; ++sub) gb[sub] = group_base(sub * S::ROWS + row);
        const uint32_t xl = (lane >> a.xs) & ((1u << a.xt) - 1u);
        uint32_t cx = 0;
#pragma unroll
        for (int q = 0; q < K; ++q)
            if ((xl >> q) & 1u) cx |= tbit[q];
        SegLanes sl;                              // the first epilogue warp stores segments
        sl.init(a.L, a.h, a.hi, lane);
        uint32_t j = 0;
        bool stop = false;
        for (unsigned long long t = first; t < tend && !stop; t += step, ++j) {
            const uint32_t ob = j % NOUT;
            float2 *out = reinterpret_cast<float2 *>(smem + S::OFF_OUT + ob * S::TILE_BYTES);
#pragma unroll
            for (uint32_t sub = 0; sub < SUB; ++sub) {
                const uint32_t js = j * SUB + sub, b = js & 1u;
                bool ok = mbar_wait_or_abort(smem_u32(&d_full[b]), (js >> 1) & 1u, abort);
                ok = ok && mbar_wait_or_abort(smem_u32(&scale_full[js & 3u]), (js >> 2) & 1u, abort);
                if (!named_bar_and(2, 256, ok)) { stop = true; break; }
                tc_fence_after();
                if (sub == 0) {
                    if (et < 32) bulk_wait_read<(int)NOUT - 1>();   // this staging tile is free
                    named_bar(2, 256);
                }
                const uint32_t gbase = gb[sub];
                const float osc = row_scale[js & 3u][row];
                const uint32_t lane_addr = tmem + b * S::ACC + ((quad * 32u) << 16) + part * HALF * 2u;
                if constexpr (XP) {
                    float2 o[HALF];
#pragma unroll
                    for (uint32_t c0 = 0; c0 < 2u * HALF; c0 += 16) {
                        float d0[16], d12[16];
                        tmem_ld16(lane_addr + c0, d0);
                        tmem_ld16(lane_addr + KD + c0, d12);
#pragma unroll
                        for (uint32_t i = 0; i < 16; i += 2) {
                            const float re = __fmaf_rn(d12[i], 1.f / 512.f, d0[i]) * osc;
                            const float im = __fmaf_rn(d12[i + 1], 1.f / 512.f, d0[i + 1]) * osc;
                            o[(c0 + i) / 2] = make_float2(re, im);
                        }
                    }
                    xor_unpermute(o, xl, a.xt);   // o[c] = member c ^ x (x < HALF)
#pragma unroll
                    for (uint32_t c = 0; c < HALF; ++c) out[gbase ^ member_off(part * HALF + c) ^ cx] = o[c];
                } else {
                    // member order: each chunk of eight members is written as soon as it is
                    // formed (fewer live registers than holding the half row)
#pragma unroll
                    for (uint32_t c0 = 0; c0 < 2u * HALF; c0 += 16) {
                        float d0[16], d12[16];
                        tmem_ld16(lane_addr + c0, d0);
                        tmem_ld16(lane_addr + KD + c0, d12);
#pragma unroll
                        for (uint32_t i = 0; i < 16; i += 2) {
                            const float re = __fmaf_rn(d12[i], 1.f / 512.f, d0[i]) * osc;
                            const float im = __fmaf_rn(d12[i + 1], 1.f / 512.f, d0[i + 1]) * osc;
                            out[gbase ^ member_off(part * HALF + (c0 + i) / 2)] = make_float2(re, im);
                        }
                    }
                }
                tc_fence_before();
                fence_proxy_async_smem();
                named_bar(2, 256);
                if (et == 0) mbar_arrive(smem_u32(&d_empty[b]));
            }
            if (stop) break;
            if (et < 32) {
                if (lane < nseg) {
                    if constexpr (SW) {
                        const int32_t row0 = (int32_t)((tile_base(sl, t) + sl.my_off) >> 4);
                        const uint32_t s0 = smem_u32(out + (size_t)lane * seg_amps);
                        for (uint32_t bx = 0; bx < a.boxes; ++bx)
                            tma_store_2d(&a.tmap, 0, row0 + (int32_t)(bx * a.box_rows), s0 + bx * a.box_rows * 128u);
                    } else {
                        bulk_s2g(psi + tile_base(sl, t) + sl.my_off, smem_u32(out + (size_t)lane * seg_amps),
                                 seg_bytes);
                    }
                }
                bulk_commit();
            }
        }
        if (et < 32) bulk_wait_all();
    }
    if (tid == 0 && abort_flag) atomicOr(a.err, 2);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == S::W_MMA) tmem_dealloc(tmem, S::TMEM_COLS);
}

// The driver's tensor-map encoder, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// `bytes` bytes at buf as a 2-D tensor of 128-byte rows (32 floats), boxes of box_rows
// rows, 128-byte swizzle in shared memory; a segment of seg_bytes (a multiple of 128) is
// `boxes` boxes.
sv_status encode_rows_map(void *buf, unsigned long long bytes, uint32_t seg_bytes, CUtensorMap *map,
                          uint32_t *box_rows, uint32_t *boxes) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return svi::set_error(SV_ERR_CUDA, "tensor-core kernel setup: cuTensorMapEncodeTiled unavailable");
    const uint32_t seg_rows = seg_bytes / 128u;
    *box_rows = std::min(seg_rows, 256u);
    *boxes = seg_rows / *box_rows;
    const cuuint64_t dims[2] = {32, bytes / 128u};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {32, *box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, buf, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return svi::set_error(SV_ERR_CUDA, "tensor-core kernel setup: cuTensorMapEncodeTiled failed (" +
                                               std::to_string((int)r) + ")");
    return SV_OK;
}

template <int K>
sv_status launch_tc_t(sv_state *s, const svi::Gate &g) {
    using S = TcShape<K, 1>;
    using S2 = TcShape<K, 2>;
    constexpr uint32_t D = S::D, KD = S::KD;
    static std::once_flag once;
    static cudaError_t init_err = cudaSuccess;
    std::call_once(once, [] {
        init_err = cudaFuncSetAttribute(apply_tc<K, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)S::SMEM);
        if (init_err == cudaSuccess)
            init_err = cudaFuncSetAttribute(apply_tc<K, true, 1>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if constexpr (K == 5) {
            if (init_err == cudaSuccess)
                init_err = cudaFuncSetAttribute(apply_tc<K, false, 2>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S2::SMEM);
            if (init_err == cudaSuccess)
                init_err = cudaFuncSetAttribute(apply_tc<K, false, 2, false, true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S2::SMEM);
        }
    });
    if (init_err != cudaSuccess)
        return svi::set_error(SV_ERR_CUDA, std::string("tensor-core kernel setup: ") +
                                               cudaGetErrorString(init_err));
    Plan p = make_plan(s->n, K, g.t, S::TB);
    // 8-byte accesses: bank pair = tile bits 0..3; targets there get lane-dependent order
    uint32_t tl = 0;
    while (tl < (uint32_t)K && p.lp[tl] < 4u) ++tl;
    // width 5 on states of at least 13 qubits: two subtiles per stage (segments twice as
    // long, half the per-stage work) with the swizzled tensor-map staging, whatever the
    // targets (no XOR member order); otherwise one subtile, XOR order for bank-bit targets
    const bool swz = K == 5 && s->n >= S2::TB;
    const bool wide = swz;
    if (wide) {
        p = make_plan(s->n, K, g.t, S2::TB);
        tl = 0;
    }
    TcArgs<K> a;
    a.box_rows = a.boxes = 0;
    if (swz) {
        const sv_status st = encode_rows_map(s->buf, 8ull << s->n, 8u << p.L, &a.tmap, &a.box_rows, &a.boxes);
        if (st != SV_OK) return st;
    }
    // R (real embedding of U) and its fixed-point slices, in FP64 on the host
    double rmax = 0.0;
    for (uint32_t i = 0; i < D * D; ++i)
        rmax = std::max(rmax, std::max(std::fabs(g.u[i].real()), std::fabs(g.u[i].imag())));
    int eb = 0;
    std::frexp(rmax, &eb);                                   // rmax < 2^eb
    const double sb = std::ldexp(1.0, 8 - eb);
    for (uint32_t n = 0; n < KD; ++n)
        for (uint32_t kk = 0; kk < KD; ++kk) {
            const svi::cplx u = g.u[(n >> 1) * D + (kk >> 1)];
            double r = ((n & 1) == (kk & 1)) ? u.real() : ((n & 1) ? u.imag() : -u.imag());
            double x = r * sb;
            const double b1 = std::nearbyint(x);
            x = (x - b1) * 512.0;
            const double b2 = std::nearbyint(x);
            x = (x - b2) * 512.0;
            const double b3 = std::nearbyint(x);
            a.b[0][n * KD + kk] = (int16_t)b1;
            a.b[1][n * KD + kk] = (int16_t)b2;
            a.b[2][n * KD + kk] = (int16_t)b3;
        }
    a.b_inv_scale = (float)std::ldexp(1.0, eb - 8);
    a.psi = s->buf;
    a.err = reinterpret_cast<int *>(s->ws + svi::WS_ERR);
    a.ntiles = p.ntiles;
    a.L = p.L;
    a.h = p.h;
    for (int j = 0; j < SV_MAX_K; ++j) a.hi[j] = p.hi[j];
    for (int j = 0; j < K; ++j) a.lp[j] = p.lp[j];
    a.xs = 4u - tl;
    a.xt = std::min(tl, (uint32_t)K - 1u);   // permute within a worker's half of the members
    const unsigned grid = (unsigned)std::min<unsigned long long>(p.ntiles, (unsigned long long)s->num_sms);
    // with eight worker warps per role the permutation costs less than even 2-way conflicts
    if (swz) {
        if constexpr (K == 5) apply_tc<K, false, 2, false, true><<<grid, S2::THREADS, S2::SMEM, s->stream>>>(a);
    } else if (a.xt >= 1) {
        apply_tc<K, true, 1><<<grid, S::THREADS, S::SMEM, s->stream>>>(a);
    } else {
        apply_tc<K, false, 1><<<grid, S::THREADS, S::SMEM, s->stream>>>(a);
    }
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

// Batched launches (sv_batch_apply): complex64 gates of width 4 or 5 on states of at least
// 12 qubits run as width-5 gates (a width-4 gate widened by an identity qubit, chosen as
// in widen_gate) with one MMA subtile per stage; each state's B is built on the device
// from the batch's FP32 matrix table.
// Batched launches use the swizzled tensor-map staging (SW), like single states.
static cudaError_t tc_batch_setup() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(apply_tc<5, false, 1, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)TcShape<5, 1, true>::SMEM);
    });
    return err;
}

// Also looks up the tensor-map encoder, so that a launch inside a stream capture finds it.
cudaError_t tc_batch_prepare() {
    const cudaError_t e = tc_batch_setup();
    if (e == cudaSuccess && !tensor_map_encoder()) return cudaErrorNotSupported;
    return e;
}

sv_status launch_tc_batch(const sv_batch_launch &L) {
    using S = TcShape<5, 1, true>;
    const cudaError_t e0 = tc_batch_prepare();
    if (e0 != cudaSuccess)
        return svi::set_error(SV_ERR_CUDA, std::string("batched tensor-core kernel setup: ") + cudaGetErrorString(e0));
    uint32_t t5[5];
    int jw = -1;
    if (L.k == 5) {
        for (int j = 0; j < 5; ++j) t5[j] = L.t[j];
    } else {
        // the identity qubit: the smallest non-target at or above bit 5, else below it
        bool used[64] = {false};
        for (uint32_t j = 0; j < 4; ++j) used[L.t[j]] = true;
        uint32_t q = 64;
        for (uint32_t c = 5; c < L.n && q == 64; ++c)
            if (!used[c]) q = c;
        for (uint32_t c = 0; c < L.n && q == 64; ++c)
            if (!used[c]) q = c;
        uint32_t m = 0;
        for (uint32_t j = 0; j < 4; ++j) {
            if (q < L.t[j] && jw < 0) { jw = (int)m; t5[m++] = q; }
            t5[m++] = L.t[j];
        }
        if (jw < 0) { jw = (int)m; t5[m++] = q; }
    }
    const Plan p = make_plan(L.n, 5, t5, S::TB);
    TcArgs<5> a;
    // the whole batch (states back to back) as one tensor; the swizzle spreads the banks
    const sv_status st = encode_rows_map(L.psi, (8ull * L.states) << L.n, 8u << p.L, &a.tmap, &a.box_rows,
                                         &a.boxes);
    if (st != SV_OK) return st;
    std::memset(a.b, 0, sizeof(a.b));
    a.b_inv_scale = 1.f;
    a.psi = L.psi;
    a.err = L.err;
    a.ntiles = p.ntiles * L.states;
    a.L = p.L;
    a.h = p.h;
    for (int j = 0; j < SV_MAX_K; ++j) a.hi[j] = p.hi[j];
    for (int j = 0; j < 5; ++j) a.lp[j] = p.lp[j];
    a.xs = 0;
    a.xt = 0;
    a.utab = static_cast<const float *>(L.utab);
    a.tiles_per_state = p.ntiles;
    a.n = L.n;
    a.kin = L.k;
    a.jw = jw;
    const unsigned grid = (unsigned)std::min<unsigned long long>(a.ntiles, (unsigned long long)L.num_sms);
    apply_tc<5, false, 1, true, true><<<grid, S::THREADS, S::SMEM, L.stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

}  // namespace svk

namespace svi {

// Width 4 and 5, and on states of at least 13 qubits every dense width (narrower gates run
// as width-5 ones, U (x) I, on the swizzled two-subtile kernel: at 30 qubits its passes
// take 2.59-2.74 ms against 2.74 for the width-2/3 CUDA-core kernel).
bool tc_eligible(const sv_state *s, const Gate &g) {
    if (s->dtype != SV_C64 || (s->policy & SV_POLICY_NO_TENSOR_CORES)) return false;
    if (g.k == 4 || g.k == 5) return s->n >= g.k + 7;
    return g.k >= 1 && s->n >= svk::TcShape<5, 2>::TB;
}

// Width-4 gates run as width-5 ones (U (x) I) where the state allows: the k = 5 kernel
// moves a tile with half the per-tile overhead of the k = 4 one for the same bytes.
sv_status launch_apply_tc(sv_state *s, const Gate &g) {
    if (g.k == 5) return svk::launch_tc_t<5>(s, g);
    if (s->n >= svk::TcShape<5, 1>::TB) return svk::launch_tc_t<5>(s, widen_gate(g, s->n, 5));
    return svk::launch_tc_t<4>(s, g);
}

}  // namespace svi
