// Two fused gates in one HBM pass (complex64, 5th-generation tensor cores).
//
// Algorithm 2 leaves a schedule of dense k-qubit gates (k <= 5), each of which costs one
// read and one write of the state when applied on its own (Eq. 10).  When two gates of
// the schedule act only on qubits of one 2^12-amplitude tile -- the index bits [0, L)
// plus the two gates' targets at or above L -- both can be applied while the tile sits
// in shared memory, so the pair costs one pass instead of two.  The arithmetic of each
// gate: per group of 32 amplitudes the real contraction v' = R v with R the real
// embedding of the (widened) 5-qubit U, on exact 9-bit fixed-point slices of A (per
// group row, x s = a1 + a2 2^-9 + a3 2^-18) and of R (R s_B = b1 + b2 2^-9 + b3 2^-18),
// with the slices kept at their scale in FP16 (a2 2^-9, a3 2^-18 ... are exact FP16
// values).  Three MMA products per K step fill three adjacent FP32 accumulators:
//     A1 [B1 B2 B3]  -> [D0 D1 D2]      (N = 192)
//     A2 [B1 B2]     ->    [D1 D2]      (N = 128)
//     A3 [B1]        ->       [D2]      (N = 64)
// so D0 = a1 b1, D1 = (a1 b2 + a2 b1) 2^-9, D2 = (a1 b3 + a2 b2 + a3 b1) 2^-18 summed
// over K = 64.  Every partial sum is a multiple of the accumulator's grid below 2^24 of
// it, so all three accumulations are exact (no truncation, no bias); the dropped terms
// sit 2^-27 below the row's largest amplitude, and out = (D0 + D1 + D2) / (s s_B) takes
// one FP32 rounding.  (Twelve MMA instructions per 128 groups, where two N = 64
// accumulators would take 24: a tcgen05.mma costs about the same time for N = 64 and
// N = 192.)  A gate narrower than 5 qubits is applied as U (x) I on tile bits it does
// not touch (the host widens it).
//
// Tile: 128 groups of 32 members = 4096 amplitudes (32 KiB), moved as 2^h contiguous
// segments of 2^L amplitudes (L >= 5, h <= 7) by 1-D bulk copies; the tile is processed
// in place: gate 0 reads the loaded stage and writes its results back into it, gate 1
// reads those and writes its own, and the stage is then stored.  To keep the roles busy
// while gate 1 of a tile waits for gate 0's last results, tiles are taken in pairs and
// the work items ordered (t, 0), (t + 1, 0), (t, 1), (t + 1, 1).
//
// One persistent CTA per SM, 18 warps, every hand-off an mbarrier:
//   warp 8               TMA: bulk loads of each tile into a ring of NS stages;
//   warps 0-7            transform: two warps per TMEM lane quadrant, one group (row of
//                        A) and half its members per thread; gather from the stage with
//                        the item's gate's target positions, the three slices in
//                        registers, then tcgen05.st into tensor memory once the previous
//                        item's MMAs have read it (A single-buffered);
//   warp 9 (one thread)  MMA issuer: 3 x 4 tcgen05.mma.kind::f16 per item with the
//                        item's gate's B, into double-buffered TMEM accumulators;
//   warps 10-17          epilogue: tcgen05.ld, combine, scatter back into the stage;
//   warp 8 also stores a tile after its last gate and reloads the stage once the store
//   has read it.  Apart from the two warps that share a row meeting once per item, the
//   warps synchronise only through mbarriers (counted arrivals), so their phases --
//   gathers, slicing, tensor-memory traffic, scatters -- overlap instead of running in
//   lockstep.
// XP: some gate of the pass has targets among tile bits 0..3; lanes then take that
// gate's members in the lane-dependent XOR order of the single-gate kernel (undone in
// registers), gates without such targets keep the plain order (runtime xt = 0).
// Every wait is bounded (2 s) and sets the abort flag; TMEM is freed on every exit.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>

#include "ptx.cuh"
#include "sv_internal.h"
#include "tc.cuh"

namespace svk {

struct Tc2Shape {
    static constexpr uint32_t K = 5;
    static constexpr uint32_t D = 32;                   // amplitudes per group
    static constexpr uint32_t KD = 64;                  // real K = N
    static constexpr uint32_t ROWS = 128;               // groups per tile (MMA M)
    static constexpr uint32_t TB = 12;                  // tile bits
    static constexpr uint32_t LMIN = 5;                 // segments of at least 256 bytes
    static constexpr uint32_t HMAX = TB - LMIN;         // high tile bits
    static constexpr uint32_t TILE_BYTES = ROWS * D * 8u;
    static constexpr uint32_t GMAX = 2;                 // gates per pass
    static constexpr uint32_t B_BYTES = KD * KD * 2u;   // one FP16 slice of B
    static constexpr uint32_t NB = 3;                   // B1, B2 2^-9, B3 2^-18
    static constexpr uint32_t B_SET = NB * B_BYTES;
    static constexpr uint32_t SBO = (KD / 8u) * 128u;
    static constexpr uint32_t NS = 5;                   // tile stages
    static constexpr uint32_t OFF_RAW = GMAX * B_SET;
    static constexpr uint32_t SMEM = OFF_RAW + NS * TILE_BYTES;
    static constexpr uint32_t ACC = 3u * KD;            // TMEM columns of one D set (D0, D1, D2)
    static constexpr uint32_t A_COLS = KD / 2u;         // TMEM columns of one A slice
    static constexpr uint32_t NA = 3;                   // A1, A2 2^-9, A3 2^-18
    static constexpr uint32_t A_SET = NA * A_COLS;      // one A buffer
    static constexpr uint32_t A_COL0 = 2u * ACC;
    static constexpr uint32_t TMEM_COLS = 512;
    static_assert(A_COL0 + A_SET <= TMEM_COLS, "TMEM layout");
    static constexpr uint32_t THREADS = 576;
    static constexpr uint32_t W_PROD = 8, W_MMA = 9, W_EPI = 10;
    static constexpr uint32_t HALF = D / 2;             // group members per worker thread
};

struct Tc2Args {
    // per gate: the three 9-bit slices of Re U and Im U (32 x 32, row-major) on the
    // gate's grid, |slice| <= 256; R (x) s_B = slices of its real embedding
    int16_t ub[Tc2Shape::GMAX][3][2][32 * 32];
    float b_inv_scale[Tc2Shape::GMAX];
    void *psi;
    int *err;
    unsigned long long ntiles;
    uint32_t L, h, G;
    uint32_t hi[Tc2Shape::HMAX];          // high tile bits (state qubits), ascending
    uint32_t lp[Tc2Shape::GMAX][5];       // each gate's targets as tile bits, ascending
    uint32_t xs[Tc2Shape::GMAX], xt[Tc2Shape::GMAX];
};

namespace {

template <int N>
__device__ __forceinline__ void xor_unpermute2(float2 (&v)[N], uint32_t x, uint32_t xt) {
    constexpr int NBITS = N >= 16 ? 4 : (N >= 8 ? 3 : (N >= 4 ? 2 : 1));
#pragma unroll
    for (int j = 0; j < NBITS; ++j) {
        if (xt > (uint32_t)j) {
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

// Three loads of 8 consecutive TMEM columns of this thread's lane (at a0, a0 + stride,
// a0 + 2 stride) and one wait.
__device__ __forceinline__ void tmem_ld8x3(uint32_t a0, uint32_t stride, float (&v)[3][8]) {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(a0), "r"(a0 + stride), "r"(a0 + 2 * stride)
        : "memory");
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[q][i] = __uint_as_float(r[8 * q + i]);
}

// max(m, |a|, |b|) in one three-input maximum (sm_100 and later).
__device__ __forceinline__ float max_abs2(float m, float a, float b) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m), "f"(fabsf(a)), "f"(fabsf(b)));
    return r;
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// The three slices of a scaled amplitude (|x scale| < 256) at their scale: a1 (an
// integer), a2 2^-9 and a3 2^-18, with |a_i| <= 256; each FP16 pair (re, im) is exact.
// Rounding to the grid 2^e (ties to even, |x| < 2^(e + 22)) adds and subtracts
// c = 1.5 2^(e + 23): the sum keeps a unit in the last place of 2^e, so it is rounded to
// that grid, and the subtraction is exact; the remainders x - a1 and (x - a1) - a2 2^-9
// are exact FP32 differences (one fused multiply-add by -1).  (re, im) go through each
// step together as one packed FP32x2 instruction.
__device__ __forceinline__ void slices(float2 v, float2 scale, uint32_t &w1, uint32_t &w2, uint32_t &w3) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 x = __fmul2_rn(v, scale);
    const float2 r1 = __fadd2_rn(__fadd2_rn(x, make_float2(12582912.f, 12582912.f)),
                                 make_float2(-12582912.f, -12582912.f));              // 1.5 2^23
    const float2 x2 = __ffma2_rn(r1, m1, x);
    const float2 r2 = __fadd2_rn(__fadd2_rn(x2, make_float2(24576.f, 24576.f)),
                                 make_float2(-24576.f, -24576.f));                    // 1.5 2^14
    const float2 x3 = __ffma2_rn(r2, m1, x2);
    const float2 r3 = __fadd2_rn(__fadd2_rn(x3, make_float2(48.f, 48.f)), make_float2(-48.f, -48.f));   // 1.5 2^5
    w1 = pack_h2(r1.x, r1.y);
    w2 = pack_h2(r2.x, r2.y);
    w3 = pack_h2(r3.x, r3.y);
}

// The tile's layout in the state (read from the kernel parameters): tile t's base
// deposits t around the high tile bits; segment q of a tile starts at base + seg_off(q).
__device__ __forceinline__ unsigned long long tile_base(const Tc2Args &a, unsigned long long t) {
    unsigned long long b = t << a.L;
#pragma unroll
    for (uint32_t j = 0; j < Tc2Shape::HMAX; ++j)
        if (j < a.h) {
            const uint32_t p = a.hi[j];
            const unsigned long long lo = b & ((1ull << p) - 1ull);
            b = ((b >> p) << (p + 1)) | lo;
        }
    return b;
}
__device__ __forceinline__ unsigned long long seg_off(const Tc2Args &a, uint32_t q) {
    unsigned long long o = 0;
#pragma unroll
    for (uint32_t j = 0; j < Tc2Shape::HMAX; ++j)
        if (j < a.h && ((q >> j) & 1u)) o |= 1ull << a.hi[j];
    return o;
}

// The gate-dependent addressing of one work item, for one thread: the group base of its
// row, the five target bits of the tile, and the lane's XOR offset.
struct GateMap {
    uint32_t gbase, cx, xl, xt;
    uint32_t tbit[5];
    __device__ __forceinline__ void init(const Tc2Args &a, uint32_t g, uint32_t row, uint32_t lane) {
        uint32_t b = row;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const uint32_t p = a.lp[g][j];
            tbit[j] = 1u << p;
            b = insert_zero32(b, p);
        }
        gbase = b;
        xt = a.xt[g];
        xl = (lane >> a.xs[g]) & ((1u << xt) - 1u);
        cx = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if ((xl >> q) & 1u) cx |= tbit[q];
    }
    __device__ __forceinline__ uint32_t member(uint32_t c) const {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if ((c >> j) & 1u) o |= tbit[j];
        return o;
    }
};

}  // namespace

template <bool XP>
__global__ void __launch_bounds__(576, 1) apply_tc2(const __grid_constant__ Tc2Args a) {
    using S = Tc2Shape;
    constexpr uint32_t KD = S::KD, NS = S::NS, HALF = S::HALF;
    extern __shared__ __align__(1024) unsigned char smem[];
    // full: a tile's load landed; gdone: gate 0's results are in the stage (8 epilogue
    // warps); tile_done: the last gate's results are in the stage (8 epilogue warps)
    __shared__ __align__(8) unsigned long long full[NS], gdone[NS], tile_done[NS];
    // a_full: 8 transform warps; a_empty, d_full: MMA commits; d_empty: 8 epilogue warps
    // (A single-buffered, D double-buffered)
    __shared__ __align__(8) unsigned long long a_full, a_empty, d_full[2], d_empty[2];
    __shared__ __align__(8) unsigned long long scale_full[4];   // 4 transform warps
    __shared__ float row_scale[4][128];
    __shared__ float max_part[2][2][128];                        // [item parity][part][row]
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    unsigned char *sB = smem;
    float2 *psi = reinterpret_cast<float2 *>(a.psi);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t seg_amps = 1u << a.L;
    const uint32_t seg_bytes = seg_amps * 8u;
    const uint32_t nseg = 1u << a.h;
    const uint32_t G = a.G;

    if (warp == S::W_MMA) {
        tmem_alloc(smem_u32(&tmem_slot), S::TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (uint32_t s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&gdone[s]), 8);
            mbar_init(smem_u32(&tile_done[s]), 8);
        }
        mbar_init(smem_u32(&a_full), 8);
        mbar_init(smem_u32(&a_empty), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&d_full[b]), 1);
            mbar_init(smem_u32(&d_empty[b]), 8);
        }
        for (int q = 0; q < 4; ++q) mbar_init(smem_u32(&scale_full[q]), 4);
        abort_flag = 0;
        fence_mbar_init();
    }
    // B of every gate: the FP16 slices B1, B2 2^-9, B3 2^-18 of R s_B in the canonical
    // K-major layout, one after the other (so [B1 B2 B3] is one 192-row operand); R[n][kk] = Re U (same parity), Im U (n odd), -Im U (n even, kk odd)
    for (uint32_t e = tid; e < G * KD * KD; e += blockDim.x) {
        const uint32_t g = e / (KD * KD), r = e % (KD * KD);
        const uint32_t n = r / KD, kk = r % KD;
        const uint32_t idx = (n >> 1) * 32u + (kk >> 1);
        const bool same = (n & 1u) == (kk & 1u);
        const int part = same ? 0 : 1;
        const int sign = (!same && !(n & 1u)) ? -1 : 1;
        const uint32_t off = g * S::B_SET + kmajor_off16(n, kk, S::SBO);
        // b1, b2 2^-9, b3 2^-18: integers below 2^9 times powers of two, exact in FP16
        *reinterpret_cast<__half *>(sB + 0 * S::B_BYTES + off) = __int2half_rn(sign * a.ub[g][0][part][idx]);
        *reinterpret_cast<__half *>(sB + 1 * S::B_BYTES + off) =
            __float2half_rn((float)(sign * a.ub[g][1][part][idx]) * (1.f / 512.f));
        *reinterpret_cast<__half *>(sB + 2 * S::B_BYTES + off) =
            __float2half_rn((float)(sign * a.ub[g][2][part][idx]) * (1.f / 262144.f));
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abort = &abort_flag;

    // This CTA's tiles: blockIdx.x + j gridDim.x, j < ntl; work items in pairs of tiles:
    // for pair p, for gate g, for the pair's tiles.
    const unsigned long long ntl =
        a.ntiles > blockIdx.x ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0ull;
    const unsigned long long npairs = (ntl + 1) / 2;

    if (warp == S::W_PROD) {
        // ------------------------------------------------------------ TMA producer
        // The stage's whole cycle: load tile j, wait until its last gate is applied, store
        // it, wait until the store has read the stage, load tile j + NS into it.
        unsigned long long off[4];
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i) off[i] = seg_off(a, lane + 32u * i);
        auto load = [&](unsigned long long j) {
            const uint32_t s = (uint32_t)(j % NS);
            const uint32_t bar = smem_u32(&full[s]);
            if (lane == 0) mbar_arrive_expect_tx(bar, S::TILE_BYTES);
            __syncwarp();
            const unsigned long long base = tile_base(a, blockIdx.x + j * gridDim.x);
            float2 *dst = reinterpret_cast<float2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
#pragma unroll
            for (uint32_t i = 0; i < 4; ++i) {
                const uint32_t q = lane + 32u * i;
                if (q < nseg)
                    bulk_g2s(smem_u32(dst + (size_t)q * seg_amps), psi + base + off[i], seg_bytes, bar);
            }
        };
        for (unsigned long long j = 0; j < ntl && j < NS; ++j) load(j);
        for (unsigned long long j = 0; j < ntl; ++j) {
            const uint32_t s = (uint32_t)(j % NS), u = (uint32_t)(j / NS);
            bool ok = true;
            if (lane == 0) ok = mbar_wait_or_abort(smem_u32(&tile_done[s]), u & 1u, abort);
            if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
            const unsigned long long base = tile_base(a, blockIdx.x + j * gridDim.x);
            const float2 *src = reinterpret_cast<const float2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
#pragma unroll
            for (uint32_t i = 0; i < 4; ++i) {
                const uint32_t q = lane + 32u * i;
                if (q < nseg) bulk_s2g(psi + base + off[i], smem_u32(src + (size_t)q * seg_amps), seg_bytes);
            }
            bulk_commit();
            if (j + NS < ntl) {
                bulk_wait_read<0>();              // the stage has been read out
                __syncwarp();
                load(j + NS);
            }
        }
        bulk_wait_all();
    } else if (warp == S::W_MMA) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            unsigned long long i = 0;
            bool stop = false;
            for (unsigned long long p = 0; p < npairs && !stop; ++p) {
                for (uint32_t g = 0; g < G && !stop; ++g) {
                    for (uint32_t q = 0; q < 2; ++q) {
                        if (2 * p + q >= ntl) break;
                        const uint32_t b = (uint32_t)i & 1u, u = (uint32_t)(i >> 1);
                        if (!mbar_wait_or_abort(smem_u32(&a_full), (uint32_t)i & 1u, abort) ||
                            !mbar_wait_or_abort(smem_u32(&d_empty[b]), (u & 1u) ^ 1u, abort)) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t A0 = tmem + S::A_COL0;
                        const uint32_t dset = tmem + b * S::ACC;
                        const uint32_t B0 = smem_u32(sB) + g * S::B_SET;
                        // A1 [B1 B2 B3] -> [D0 D1 D2], A2 [B1 B2] -> [D1 D2], A3 B1 -> D2;
                        // B from its first slice, N rows (the slices are consecutive)
#pragma unroll
                        for (uint32_t pr = 0; pr < 3; ++pr) {
                            const uint32_t idesc = idesc_f16(S::ROWS, (3u - pr) * KD);
#pragma unroll
                            for (uint32_t ks = 0; ks < KD / 16; ++ks)
                                mma_f16_tmem_a(dset + pr * KD, A0 + pr * S::A_COLS + ks * 8u,
                                               smem_desc(B0 + ks * 256u, 128u, S::SBO), idesc,
                                               (pr == 0 && ks == 0) ? 0u : 1u);
                        }
                        mma_commit(smem_u32(&a_empty));
                        mma_commit(smem_u32(&d_full[b]));
                        ++i;
                    }
                }
            }
        }
    } else if (warp < S::W_PROD) {
        // ------------------------------------------------------------ transform
        // Warps quad and quad + 4 share the rows of TMEM lane quadrant `quad` (one group per
        // thread, half its members each) and meet once per item to combine their halves'
        // largest components; otherwise every warp runs on its own.
        const uint32_t quad = warp & 3u;
        const uint32_t row = quad * 32u + lane;
        const uint32_t part = warp >> 2;
        unsigned long long i = 0;
        bool stop = false, bad = false;
        for (unsigned long long p = 0; p < npairs && !stop; ++p) {
            for (uint32_t g = 0; g < G && !stop; ++g) {
                GateMap gm;
                gm.init(a, g, row, lane);
                for (uint32_t q = 0; q < 2; ++q) {
                    const unsigned long long j = 2 * p + q;
                    if (j >= ntl) break;
                    const uint32_t s = (uint32_t)(j % NS), u = (uint32_t)(j / NS);
                    // gate 0 reads the loaded tile, gate 1 the results of gate 0; a warp that
                    // gave up earlier (bad) still meets its partner here, so both stop
                    bool ok = !bad && mbar_wait_or_abort(smem_u32(g == 0 ? &full[s] : &gdone[s]), u & 1u, abort);
                    const float2 *rs = reinterpret_cast<const float2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
                    float2 v[HALF];
                    float m = 0.f;
                    if (ok) {
#pragma unroll
                        for (uint32_t c = 0; c < HALF; ++c) {
                            const uint32_t mo = gm.member(part * HALF + c);
                            v[c] = rs[gm.gbase | (XP ? (mo ^ gm.cx) : mo)];
                            m = max_abs2(m, v[c].x, v[c].y);
                        }
                    }
                    max_part[i & 1u][part][row] = m;
                    if (!named_bar_and(3u + quad, 64, ok)) { stop = true; break; }
                    m = fmaxf(max_part[i & 1u][0][row], max_part[i & 1u][1][row]);
                    int ex = 0;
                    frexpf(m, &ex);                   // m < 2^ex (m = 0: ex = 0)
                    ex = max(ex, -100);
                    const float sc = ldexpf(1.f, 8 - ex);      // |x * sc| < 256
                    const float2 scale = make_float2(sc, sc);
                    if constexpr (XP) xor_unpermute2(v, gm.xl, gm.xt);
                    // the first eight members' slices before waiting for the A buffer, the
                    // other eight after (fewer live registers)
                    uint32_t w1[8], w2[8], w3[8];
#pragma unroll
                    for (uint32_t c = 0; c < 8; ++c) slices(v[c], scale, w1[c], w2[c], w3[c]);
                    // the single A buffer: free once the MMAs of item i - 1 completed
                    if (!mbar_wait_or_abort(smem_u32(&a_empty), ((uint32_t)i & 1u) ^ 1u, abort)) {
                        bad = true;
                        ++i;
                        continue;
                    }
                    tc_fence_after();
                    // slot i & 3 was last read by the epilogue of item i - 4, before it released
                    // the accumulators that the MMAs of item i - 2 then wrote; those completed
                    // before the MMAs of item i - 1, whose completion released a_empty
                    if (part == 0) row_scale[i & 3u][row] = ldexpf(a.b_inv_scale[g], ex - 8);
                    const uint32_t arow = tmem + S::A_COL0 + ((quad * 32u) << 16) + part * HALF;
                    tmem_st8_async(arow, w1);
                    tmem_st8_async(arow + S::A_COLS, w2);
                    tmem_st8_async(arow + 2 * S::A_COLS, w3);
#pragma unroll
                    for (uint32_t c = 0; c < 8; ++c) slices(v[8 + c], scale, w1[c], w2[c], w3[c]);
                    tmem_st8_async(arow + 8, w1);
                    tmem_st8_async(arow + S::A_COLS + 8, w2);
                    tmem_st8_async(arow + 2 * S::A_COLS + 8, w3);
                    tmem_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(smem_u32(&a_full));
                        if (part == 0) mbar_arrive(smem_u32(&scale_full[i & 3u]));
                    }
                    ++i;
                }
            }
        }
    } else if (warp >= S::W_EPI) {
        // ------------------------------------------------------------ epilogue
        // Every warp on its own: its quadrant's rows, half the accumulator columns.
        const uint32_t quad = warp & 3u;
        const uint32_t row = quad * 32u + lane;
        const uint32_t part = (warp - S::W_EPI) >> 2;
        unsigned long long i = 0;
        bool stop = false;
        for (unsigned long long p = 0; p < npairs && !stop; ++p) {
            for (uint32_t g = 0; g < G && !stop; ++g) {
                GateMap gm;
                gm.init(a, g, row, lane);
                for (uint32_t q = 0; q < 2; ++q) {
                    const unsigned long long j = 2 * p + q;
                    if (j >= ntl) break;
                    const uint32_t s = (uint32_t)(j % NS);
                    const uint32_t b = (uint32_t)i & 1u;
                    bool ok = mbar_wait_or_abort(smem_u32(&d_full[b]), (uint32_t)(i >> 1) & 1u, abort);
                    ok = ok && mbar_wait_or_abort(smem_u32(&scale_full[i & 3u]), (uint32_t)(i >> 2) & 1u, abort);
                    if (!__all_sync(0xffffffffu, ok)) { stop = true; break; }
                    tc_fence_after();
                    float2 *st = reinterpret_cast<float2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
                    const float osc = row_scale[i & 3u][row];
                    const float2 osc2 = make_float2(osc, osc);
                    const uint32_t lane_addr = tmem + b * S::ACC + ((quad * 32u) << 16) + part * HALF * 2u;
                    float2 o[HALF];
#pragma unroll
                    for (uint32_t c0 = 0; c0 < 2u * HALF; c0 += 8) {
                        float d[3][8];
                        tmem_ld8x3(lane_addr + c0, KD, d);
#pragma unroll
                        for (uint32_t e = 0; e < 8; e += 2) {
                            const float2 s12 = __fadd2_rn(make_float2(d[1][e], d[1][e + 1]),
                                                          make_float2(d[2][e], d[2][e + 1]));
                            const float2 sum = __fadd2_rn(make_float2(d[0][e], d[0][e + 1]), s12);
                            o[(c0 + e) / 2] = __fmul2_rn(sum, osc2);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&d_empty[b]));
                    if constexpr (XP) xor_unpermute2(o, gm.xl, gm.xt);
                    // in place: the transform of this item read these amplitudes before
                    // its A buffer, and so these accumulators, could be produced
#pragma unroll
                    for (uint32_t c = 0; c < HALF; ++c) {
                        const uint32_t mo = gm.member(part * HALF + c);
                        st[gm.gbase | (XP ? (mo ^ gm.cx) : mo)] = o[c];
                    }
                    fence_proxy_async_smem();         // the producer's bulk store reads them
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(g + 1 < G ? &gdone[s] : &tile_done[s]));
                    ++i;
                }
            }
        }
    }
    if (tid == 0 && abort_flag) atomicOr(a.err, 2);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == S::W_MMA) tmem_dealloc(tmem, S::TMEM_COLS);
}

}  // namespace svk

namespace svi {

namespace {

// Tile geometry of a pass over the union of the gates' targets: the largest L with
// L + #{targets >= L} <= 12.
uint32_t pass_low_bits(uint32_t n, const uint32_t *u, uint32_t nu) {
    const uint32_t TB = svk::Tc2Shape::TB;
    for (uint32_t L = std::min(TB, n);; --L) {
        uint32_t h = 0;
        for (uint32_t j = 0; j < nu; ++j) h += u[j] >= L;
        if (L + h <= TB || L == 0) return L + h <= TB ? L : 0;
    }
}

uint32_t union_targets(const Gate &g0, const Gate &g1, uint32_t *u) {
    uint32_t m = 0;
    for (uint32_t j = 0; j < g0.k; ++j) u[m++] = g0.t[j];
    for (uint32_t j = 0; j < g1.k; ++j) {
        bool seen = false;
        for (uint32_t i = 0; i < g0.k; ++i) seen = seen || g0.t[i] == g1.t[j];
        if (!seen) u[m++] = g1.t[j];
    }
    std::sort(u, u + m);
    return m;
}

}  // namespace

bool tc2_pair_fits(const sv_state *s, const Gate &g0, const Gate &g1) {
    if (s->dtype != SV_C64 || s->n < svk::Tc2Shape::TB + 1) return false;
    uint32_t u[2 * SV_MAX_K];
    const uint32_t m = union_targets(g0, g1, u);
    return pass_low_bits(s->n, u, m) >= svk::Tc2Shape::LMIN;
}

// Both gates of a pair as 5-qubit gates on qubits of the pass's tile (identity on the
// added ones, taken from the tile's bits 4 and up where possible, so that the widening
// adds no targets among the bank-selecting bits), then one launch.
sv_status launch_apply_tc2(sv_state *s, const Gate &g0_in, const Gate &g1_in) {
    using S = svk::Tc2Shape;
    static std::once_flag once;
    static cudaError_t init_err = cudaSuccess;
    std::call_once(once, [] {
        init_err = cudaFuncSetAttribute(svk::apply_tc2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)S::SMEM);
        if (init_err == cudaSuccess)
            init_err = cudaFuncSetAttribute(svk::apply_tc2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)S::SMEM);
    });
    if (init_err != cudaSuccess)
        return set_error(SV_ERR_CUDA, std::string("two-gate tensor-core kernel setup: ") + cudaGetErrorString(init_err));
    uint32_t u[2 * SV_MAX_K];
    const uint32_t m = union_targets(g0_in, g1_in, u);
    const uint32_t L = pass_low_bits(s->n, u, m);
    if (s->dtype != SV_C64 || s->n < S::TB + 1 || L < S::LMIN)
        return set_error(SV_ERR_ARG, "two-gate pass: the gates do not fit one tile");
    // tile bits -> state qubits: [0, L) then the high targets
    uint32_t tq[S::TB];
    uint32_t h = 0;
    for (uint32_t q = 0; q < L; ++q) tq[q] = q;
    svk::Tc2Args *ap = new svk::Tc2Args;
    std::unique_ptr<svk::Tc2Args> hold(ap);
    svk::Tc2Args &a = *ap;
    std::memset(&a, 0, sizeof(a));
    for (uint32_t j = 0; j < m; ++j)
        if (u[j] >= L) {
            a.hi[h] = u[j];
            tq[L + h] = u[j];
            ++h;
        }
    const Gate *gin[2] = {&g0_in, &g1_in};
    bool bank = false;
    for (uint32_t g = 0; g < 2; ++g) {
        // widen to 5 qubits with tile qubits the gate does not touch, highest first
        Gate w;
        if (gin[g]->k == 5) {
            w = *gin[g];
        } else {
            bool used[64] = {false};
            for (uint32_t j = 0; j < gin[g]->k; ++j) used[gin[g]->t[j]] = true;
            uint32_t qs[SV_MAX_K];
            uint32_t c = gin[g]->k;
            for (uint32_t j = 0; j < gin[g]->k; ++j) qs[j] = gin[g]->t[j];
            for (int b = (int)(L + h) - 1; b >= 0 && c < 5; --b)
                if (!used[tq[b]]) {
                    used[tq[b]] = true;
                    qs[c++] = tq[b];
                }
            std::sort(qs, qs + 5);
            w = widen_gate_on(*gin[g], qs, 5);
        }
        // target positions in the tile
        uint32_t tl = 0;
        for (uint32_t j = 0; j < 5; ++j) {
            uint32_t pos = w.t[j];
            if (w.t[j] >= L)
                for (uint32_t i = 0; i < h; ++i)
                    if (a.hi[i] == w.t[j]) pos = L + i;
            a.lp[g][j] = pos;
            tl += pos < 4u;
        }
        a.xs[g] = 4u - tl;
        a.xt[g] = std::min(tl, 4u);
        bank = bank || tl > 0;
        // slices of Re U and Im U on the gate's grid (max |entry| of R < 2^eb)
        double rmax = 0.0;
        for (const cplx &z : w.u) rmax = std::max(rmax, std::max(std::fabs(z.real()), std::fabs(z.imag())));
        int eb = 0;
        std::frexp(rmax, &eb);
        const double sb = std::ldexp(1.0, 8 - eb);
        for (uint32_t e = 0; e < 32 * 32; ++e)
            for (int part = 0; part < 2; ++part) {
                double x = (part == 0 ? w.u[e].real() : w.u[e].imag()) * sb;
                const double b1 = std::nearbyint(x);
                x = (x - b1) * 512.0;
                const double b2 = std::nearbyint(x);
                x = (x - b2) * 512.0;
                const double b3 = std::nearbyint(x);
                a.ub[g][0][part][e] = (int16_t)b1;
                a.ub[g][1][part][e] = (int16_t)b2;
                a.ub[g][2][part][e] = (int16_t)b3;
            }
        a.b_inv_scale[g] = (float)std::ldexp(1.0, eb - 8);
    }
    a.psi = s->buf;
    a.err = reinterpret_cast<int *>(s->ws + WS_ERR);
    a.L = L;
    a.h = h;
    a.G = 2;
    a.ntiles = 1ull << (s->n - S::TB);
    const unsigned grid = (unsigned)std::min<unsigned long long>(a.ntiles, (unsigned long long)s->num_sms);
    if (bank) svk::apply_tc2<true><<<grid, S::THREADS, S::SMEM, s->stream>>>(a);
    else svk::apply_tc2<false><<<grid, S::THREADS, S::SMEM, s->stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

}  // namespace svi
