// Gates in complex128 on the 5th-generation tensor cores (tcgen05), to FP64 accuracy.
//
// As in the complex64 kernel, a tile of 128 groups of 2^4 amplitudes is the real GEMM
// D[128 x 32] = A[128 x 32] R^T (R = real embedding of the 16 x 16 gate, Eq. 3), but every
// operand is cut into six exact FP16 digits (fixed_point.h): per row of A on the grid of
// the row's largest exponent, for R on the grid of its largest entry,
//     A = sum_i A_i 2^(-9 i),  R = sum_j B_j 2^(-9 j),  i, j = 0..5, |A_i|, |B_j| <= 256.
// Level s collects the digit pairs with i + j = s; with 32 products of at most 2^16 per
// pair, the levels s = 0..3 (1, 2, 3, 4 pairs) stay below 2^24 and are accumulated
// EXACTLY by the FP32 tensor-core accumulators:
//     D0 = L0, D1 = L1, D2 = L2, D3 = L3,
//     D45 = L4 + 2^-9 L5   (with the B_j 2^-9 copies; its rounding sits 2^-45 below the
//                           leading level).
// Levels 6..10 are dropped (below 2^-46 of the row's largest term).  The epilogue
// converts the accumulators to integers, forms Z = L0 2^40 + L1 2^31 + L2 2^22 + L3 2^13 +
// rint(16 D45) in 64 bits and builds the nearest double of Z 2^p with integer operations
// (an identity gate returns its input bit for bit).
// 21 digit products per tile; the split and the products never touch the FP64 pipe (this
// GPU runs it at about 1/64 of the FP32 rate), only the final int64 -> double conversion
// of each output does, which balances the integer and FP64 pipes.
//
// Gates on fewer than four qubits are widened to four (U (x) I on extra qubits chosen
// above bit 4, so a warp's rows stay contiguous in shared memory).
//
// Roles and pipelines follow the complex64 kernel, with twice the integer workers: warps
// 0-7 digit transform into TMEM (tcgen05.st), warp 8 TMA producer (lane i copies segment
// i), warp 9 lane 0 the MMA issuer, warps 10-17 the epilogue with bulk stores; A and D
// double-buffered in TMEM (2 x 96 + 2 x 160 = 512 columns); every wait bounded with a
// shared abort flag.
#include <cuda_fp16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "fixed_point.h"
#include "plan.h"
#include "ptx.cuh"
#include "sv_internal.h"
#include "tc.cuh"

namespace svk {

// SUB: MMA subtiles (128 groups each) per TMA stage.  SUB = 2 doubles the contiguous
// segments of launches whose targets sit above the low index bits (4 KiB instead of 2).
template <int SUB = 1>
struct Tc64S {
    static constexpr uint32_t K = 4;
    static constexpr uint32_t D = 16;                     // amplitudes per group
    static constexpr uint32_t KD = 32;                    // real K = N
    static constexpr uint32_t ROWS = 128;                 // groups per MMA subtile (MMA M)
    static constexpr uint32_t TB = 11 + (SUB == 2 ? 1u : 0u);   // tile bits
    static constexpr uint32_t TILE_BYTES = SUB * ROWS * D * 16u;  // 32 or 64 KB
    static constexpr uint32_t B_BYTES = KD * KD * 2u;     // one FP16 digit slice of R
    static constexpr uint32_t NB = 12;                    // B_j and B_j 2^-9, j = 0..5
    static constexpr uint32_t SBO = (KD / 8u) * 128u;
    static constexpr uint32_t NS = SUB == 2 ? 2u : 4u;    // raw stages
    static constexpr uint32_t NOUT = SUB == 2 ? 1u : 2u;  // output staging tiles
    static constexpr uint32_t NACC = 5;                   // D0, D1, D2, D3, D45
    static constexpr uint32_t ACC = NACC * KD;            // TMEM columns of one D set
    static constexpr uint32_t A_COLS = KD / 2u;           // TMEM columns of one A digit slice
    static constexpr uint32_t A_SET = 6u * A_COLS;        // one A buffer (six slices)
    static constexpr uint32_t A_COL0 = 2u * ACC;
    static constexpr uint32_t TMEM_COLS = 512;
    static_assert(A_COL0 + 2u * A_SET <= TMEM_COLS, "TMEM layout");
    static constexpr uint32_t OFF_RAW = NB * B_BYTES;
    static constexpr uint32_t OFF_OUT = OFF_RAW + NS * TILE_BYTES;
    static constexpr uint32_t SMEM = OFF_OUT + NOUT * TILE_BYTES;
    static constexpr uint32_t THREADS = 576;              // 18 warps
    // warps 0-7 transform, 8 producer, 9 MMA issuer, 10-17 epilogue
    static constexpr uint32_t W_PROD = 8, W_MMA = 9, W_EPI = 10;
};
using Tc64 = Tc64S<1>;

struct Tc64Args {
    // swizzled launches (SW): the state as a 2-D tensor of 128-byte rows (8 amplitudes),
    // `boxes` boxes of box_rows rows per segment, 128-byte swizzle in shared memory
    CUtensorMap tmap;
    uint32_t box_rows, boxes;
    int16_t b[6][32 * 32];   // digits of R (row-major n x kk), most significant first
    int b_exp;               // max |R| < 2^b_exp
    void *psi;
    int *err;
    unsigned long long ntiles;
    uint32_t L, h;
    uint32_t hi[SV_MAX_K];
    uint32_t lp[4];
    // bank-conflict avoidance: the xt (<= 2) lowest targets sit at tile bits below 3; lane
    // l takes the members of each group of four in the order c ^ x(l), x(l) = (l >> xs) &
    // (2^xt - 1)
    uint32_t xs, xt;
};

// v[c] <- v[c ^ x] for c < 4 and the low xt (<= 2) bits of x.
template <typename T, typename Sel>
__device__ __forceinline__ void xor_unpermute4(T (&v)[4], uint32_t x, uint32_t xt, Sel sel) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        if (xt > (uint32_t)j) {                       // uniform over the launch
            const bool f = (x >> j) & 1u;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c & (1 << j)) continue;
                const T lo = v[c], hi = v[c | (1 << j)];
                v[c] = sel(f, hi, lo);
                v[c | (1 << j)] = sel(f, lo, hi);
            }
        }
    }
}

__device__ __forceinline__ uint4 sel_u4(bool f, uint4 a, uint4 b) {
    return make_uint4(f ? a.x : b.x, f ? a.y : b.y, f ? a.z : b.z, f ? a.w : b.w);
}

__device__ __forceinline__ double2 sel_d2(bool f, double2 a, double2 b) {
    return make_double2(f ? a.x : b.x, f ? a.y : b.y);
}

// Digit-pair word -> FP16 pair of digits: the patterns read 2048 + 2u, and
// (2048 + 2u) 0.5 - 1280 = u - 256 is exact in one half2 multiply-add.
__device__ __forceinline__ uint32_t digit_pair(uint32_t word) {
    const __half2 h = __hfma2(*reinterpret_cast<const __half2 *>(&word), __float2half2_rn(0.5f),
                              __float2half2_rn(-1280.f));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Levels as integers (L0, L1 below 2^22 by the bit-pattern trick, the others by
// conversion; 16 D45 below 2^28), Z = L0 2^40 + L1 2^31 + L2 2^22 + L3 2^13 + rint(16 D45)
// in 64 bits, and the nearest double of Z 2^p.  The int64 -> double conversion runs on the
// FP64 pipe, which the rest of the kernel leaves idle: it rounds to nearest even exactly
// like fxp::assemble_words (the integer-pipe form, about 30 instructions), and the scaling
// by 2^p is an add to the exponent field while the result stays normal.  Measured at 28
// qubits: 2.55 -> 2.09 ms per pass (the integer ALU pipe was the bound).
__device__ __forceinline__ double combine_levels(float f0, float f1, float f2, float f3, float f45,
                                                 int p) {
    const long long z = (long long)__float2int_rn(f45 * 16.f) + (long long)__float2int_rn(f3) * (1ll << 13) +
                        (long long)__float2int_rn(f2) * (1ll << 22) +
                        (long long)fxp::small_float_to_int(f1) * (1ll << 31) +
                        (long long)fxp::small_float_to_int(f0) * (1ll << 40);
    if (z == 0) return 0.0;
    const long long b = __double_as_longlong(__ll2double_rn(z));
    const int e = (int)((b >> 52) & 0x7FF) + p;
    if (e < 1 || e > 2046) return fxp::assemble_slow(z, p);
    return __longlong_as_double(b + ((long long)p << 52));
}

// XP (not launched: two bank-bit targets now take the swizzled staging, SW): the launch
// has targets among tile bits 0..2 and takes members in the lane's XOR
// order; otherwise no permutation code at all.  The pipelines count tiles (j: raw stage,
// output staging) and MMA subtiles (js = j SUB + sub: A and D buffers, row exponents).
// 16-byte elements: the 128-byte swizzle XORs the 16-byte chunk (index bits 0-2) with the
// 128-byte row within each 1 KiB (index bits 3-5); linear over XOR, its own inverse.
__device__ __forceinline__ uint32_t swz128_16(uint32_t f) { return f ^ ((f >> 3) & 7u); }

// SW: tiles move by 2-D tensor-map copies with the 128-byte swizzle and the roles address
// them through it, so a warp's lanes reach different banks whatever the targets (no XOR
// member order: XP = false).  The swizzle is applied to the group base and the target
// bits, which then combine by XOR.
template <bool XP, int SUB = 1, bool SW = false>
__global__ void __launch_bounds__(576, 1) apply_tc64(const __grid_constant__ Tc64Args a) {
    using S = Tc64S<SUB>;
    constexpr uint32_t KD = S::KD, NS = S::NS, NOUT = S::NOUT;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long full[NS], empty[NS];
    __shared__ __align__(8) unsigned long long a_full[2], a_empty[2], d_full[2], d_empty[2];
    __shared__ __align__(8) unsigned long long scale_full[4];   // row exponents, tile j -> j & 3
    __shared__ int row_exp[4][128];
    __shared__ uint32_t emax_part[2][128];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    unsigned char *sB = smem;
    double2 *psi = reinterpret_cast<double2 *>(a.psi);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const uint32_t seg_amps = 1u << a.L;
    const uint32_t seg_bytes = seg_amps * 16u;
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
        abort_flag = 0;
        fence_mbar_init();
    }
    for (uint32_t e = tid; e < KD * KD; e += blockDim.x) {
        const uint32_t n = e / KD, kk = e % KD, off = kmajor_off16(n, kk, S::SBO);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            *reinterpret_cast<__half *>(sB + j * S::B_BYTES + off) = __int2half_rn(a.b[j][e]);
            // exact: an integer of at most 9 bits times 2^-9
            *reinterpret_cast<__half *>(sB + (6 + j) * S::B_BYTES + off) =
                __float2half_rn((float)a.b[j][e] * (1.f / 512.f));
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abort = &abort_flag;
    const unsigned long long first = blockIdx.x, step = gridDim.x;

    auto group_base = [&](uint32_t row) {
        uint32_t g = row;
#pragma unroll
        for (int j = 0; j < 4; ++j) g = insert_zero32(g, a.lp[j]);
        return SW ? swz128_16(g) : g;
    };
    // tile offset of target j (swizzled with SW; four registers), and of group member c:
    // the XOR of the offsets of its set bits; a member's index is group base XOR offset
    uint32_t tb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tb[j] = SW ? swz128_16(1u << a.lp[j]) : 1u << a.lp[j];
    auto member_off = [&](uint32_t c) {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((c >> j) & 1u) o ^= tb[j];
        return o;
    };

    if (warp == S::W_PROD) {
        // ------------------------------------------------------------ TMA producer
        SegLanes sl;
        sl.init(a.L, a.h, a.hi, lane);
        uint32_t j = 0;
        for (unsigned long long t = first; t < a.ntiles; t += step, ++j) {
            const uint32_t s = j % NS, u = j / NS;
            bool ok = true;
            if (lane == 0) ok = mbar_wait_or_abort(smem_u32(&empty[s]), (u & 1u) ^ 1u, abort);
            if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
            const uint32_t bar = smem_u32(&full[s]);
            if (lane == 0) mbar_arrive_expect_tx(bar, S::TILE_BYTES);
            __syncwarp();
            if (lane < nseg) {
                double2 *dst = reinterpret_cast<double2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
                if constexpr (SW) {
                    // segment = `boxes` boxes of box_rows 128-byte rows (8 amplitudes each)
                    const int32_t row0 = (int32_t)((sl.base(t) + sl.my_off) >> 3);
                    const uint32_t d0 = smem_u32(dst + (size_t)lane * seg_amps);
                    for (uint32_t bx = 0; bx < a.boxes; ++bx)
                        tma_load_2d(d0 + bx * a.box_rows * 128u, &a.tmap, 0, row0 + (int32_t)(bx * a.box_rows), bar);
                } else {
                    bulk_g2s(smem_u32(dst + (size_t)lane * seg_amps), psi + sl.base(t) + sl.my_off,
                             seg_bytes, bar);
                }
            }
        }
    } else if (warp == S::W_MMA) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(S::ROWS, KD);
            const uint32_t B0 = smem_u32(sB);
            const unsigned long long nsub = a.ntiles > first
                                                ? ((a.ntiles - first + step - 1) / step) * SUB : 0;
            for (unsigned long long js = 0; js < nsub; ++js) {
                const uint32_t b = (uint32_t)js & 1u, u = (uint32_t)(js >> 1);
                if (!mbar_wait_or_abort(smem_u32(&a_full[b]), u & 1u, abort)) break;
                if (!mbar_wait_or_abort(smem_u32(&d_empty[b]), (u & 1u) ^ 1u, abort)) break;
                tc_fence_after();
                const uint32_t A0 = tmem + S::A_COL0 + b * S::A_SET;
                const uint32_t dset = tmem + b * S::ACC;
                // (accumulator, A digit, B slice); slices 6 + j hold B_j 2^-9
                const uint32_t prod[21][3] = {
                    {0, 0, 0},
                    {1, 0, 1}, {1, 1, 0},
                    {2, 0, 2}, {2, 1, 1}, {2, 2, 0},
                    {3, 0, 3}, {3, 1, 2}, {3, 2, 1}, {3, 3, 0},
                    {4, 0, 4}, {4, 1, 3}, {4, 2, 2}, {4, 3, 1}, {4, 4, 0},
                    {4, 0, 11}, {4, 1, 10}, {4, 2, 9}, {4, 3, 8}, {4, 4, 7}, {4, 5, 6}};
#pragma unroll
                for (int p = 0; p < 21; ++p) {
                    const uint32_t acc = prod[p][0];
                    const uint32_t Aa = A0 + prod[p][1] * S::A_COLS;
                    const uint32_t Bb = B0 + prod[p][2] * S::B_BYTES;
                    const bool first_in_acc = (p == 0 || p == 1 || p == 3 || p == 6 || p == 10);
#pragma unroll
                    for (uint32_t ks = 0; ks < KD / 16; ++ks)
                        mma_f16_tmem_a(dset + acc * KD, Aa + ks * 8u,
                                       smem_desc(Bb + ks * 256u, 128u, S::SBO), idesc,
                                       (first_in_acc && ks == 0) ? 0u : 1u);
                }
                mma_commit(smem_u32(&a_empty[b]));
                mma_commit(smem_u32(&d_full[b]));
            }
        }
    } else if (warp < S::W_PROD) {
        // ------------------------------------------------------------ digit transform
        // Two warps per TMEM lane quadrant: warp w takes rows 32 (w & 3) .. + 31 and
        // group members 8 (w >> 2) .. + 7.  Rolled loops over four members at a time keep
        // the code small (the roles run different code on every SM sub-partition).
        const uint32_t row = (warp & 3u) * 32u + lane;
        const uint32_t part = warp >> 2;
        const uint32_t lo_off[4] = {0u, tb[0], tb[1], tb[0] ^ tb[1]};
        const uint32_t xl = (lane >> a.xs) & ((1u << a.xt) - 1u);
        const uint32_t cx = ((xl & 1u) << a.lp[0]) | (((xl >> 1) & 1u) << a.lp[1]);
        uint32_t j = 0;
        bool stop = false;
        for (unsigned long long t = first; t < a.ntiles && !stop; t += step, ++j) {
            const uint32_t s = j % NS;
            const bool okf = mbar_wait_or_abort(smem_u32(&full[s]), (j / NS) & 1u, abort);
            const double2 *rs = reinterpret_cast<const double2 *>(smem + S::OFF_RAW + s * S::TILE_BYTES);
#pragma unroll 1
          for (uint32_t sub = 0; sub < (uint32_t)SUB; ++sub) {
            const uint32_t js = j * SUB + sub;
            const uint32_t gbase = group_base(sub * S::ROWS + row);
            const uint32_t ab = js & 1u;
            const bool ok = okf && mbar_wait_or_abort(smem_u32(&a_empty[ab]), ((js >> 1) & 1u) ^ 1u, abort);
            // the row's largest exponent field: each half over its members (high words)
            uint32_t em = 0;                      // largest |high word|: its exponent field
#pragma unroll
            for (uint32_t c = 0; c < 8; ++c) {
                const uint32_t *w = reinterpret_cast<const uint32_t *>(
                    rs + (gbase ^ (XP ? (member_off(part * 8u + c) ^ cx) : member_off(part * 8u + c))));
                em = max(em, max(w[1] & 0x7FFFFFFFu, w[3] & 0x7FFFFFFFu));
            }
            emax_part[part][row] = max(em >> 20, 1u);
            if (!named_bar_and(1, 256, ok)) { stop = true; break; }
            tc_fence_after();
            const uint32_t emax = max(emax_part[0][row], emax_part[1][row]);
            // slot js & 3 was last read by the epilogue of subtile js - 4, which finished
            // before the MMAs of subtile js - 2 were issued, whose completion released
            // a_empty[ab]
            if (part == 0) row_exp[js & 3u][row] = (int)emax;
            const uint32_t arow = tmem + S::A_COL0 + ab * S::A_SET + (((warp & 3u) * 32u) << 16);
#pragma unroll 1
            for (uint32_t c0 = part * 8u; c0 < part * 8u + 8u; c0 += 4) {
                const uint32_t hoff = gbase ^ (((c0 >> 2) & 1u) ? tb[2] : 0u) ^ (((c0 >> 3) & 1u) ? tb[3] : 0u);
                uint32_t w[6][4];
                uint4 va[4];
#pragma unroll
                for (uint32_t c = 0; c < 4; ++c)
                    va[c] = *reinterpret_cast<const uint4 *>(rs + (hoff ^ (XP ? (lo_off[c] ^ cx) : lo_off[c])));
                if constexpr (XP) xor_unpermute4(va, xl, a.xt, sel_u4);
#pragma unroll
                for (uint32_t c = 0; c < 4; ++c) {
                    const uint4 v = va[c];
                    uint32_t rh, rl, ih, il, t[6];
                    fxp::offset_fixed(v.y, v.x, emax, rh, rl);
                    fxp::offset_fixed(v.w, v.z, emax, ih, il);
                    fxp::digit_pair_words(rh, rl, ih, il, t);
#pragma unroll
                    for (int i = 0; i < 6; ++i) w[i][c] = digit_pair(t[i]);
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) tmem_st4_async(arow + i * S::A_COLS + c0, w[i]);
            }
            fence_proxy_async_smem();             // reads of the raw stage before its refill
            tmem_wait_st();
            tc_fence_before();
            named_bar(1, 256);                    // also: emax_part is free for the next subtile
            if (tid == 0) {
                if (sub == (uint32_t)SUB - 1u) mbar_arrive(smem_u32(&empty[s]));
                mbar_arrive(smem_u32(&a_full[ab]));
                mbar_arrive(smem_u32(&scale_full[js & 3u]));
            }
          }
        }
    } else if (warp >= S::W_EPI) {
        // ------------------------------------------------------------ epilogue
        // Two warps per lane quadrant, each over 16 of the 32 accumulator columns.
        const uint32_t quad = warp & 3u;
        const uint32_t row = quad * 32u + lane;
        const uint32_t et = tid - S::W_EPI * 32u;    // 0..255
        const uint32_t part = et >> 7;
        const uint32_t lo_off[4] = {0u, tb[0], tb[1], tb[0] ^ tb[1]};
        const uint32_t xl = (lane >> a.xs) & ((1u << a.xt) - 1u);
        const uint32_t cx = ((xl & 1u) << a.lp[0]) | (((xl >> 1) & 1u) << a.lp[1]);
        SegLanes sl;
        sl.init(a.L, a.h, a.hi, lane);
        uint32_t j = 0;
        bool stop = false;
        for (unsigned long long t = first; t < a.ntiles && !stop; t += step, ++j) {
            const uint32_t ob = j % NOUT;
            double2 *out = reinterpret_cast<double2 *>(smem + S::OFF_OUT + ob * S::TILE_BYTES);
#pragma unroll 1
          for (uint32_t sub = 0; sub < (uint32_t)SUB; ++sub) {
            const uint32_t js = j * SUB + sub, b = js & 1u;
            const uint32_t gbase = group_base(sub * S::ROWS + row);
            bool ok = mbar_wait_or_abort(smem_u32(&d_full[b]), (js >> 1) & 1u, abort);
            ok = ok && mbar_wait_or_abort(smem_u32(&scale_full[js & 3u]), (js >> 2) & 1u, abort);
            if (!named_bar_and(2, 256, ok)) { stop = true; break; }
            tc_fence_after();
            if (sub == 0) {
                if (et < 32) bulk_wait_read<(int)NOUT - 1>();   // this staging tile is free
                named_bar(2, 256);
            }
            const int p = row_exp[js & 3u][row] + a.b_exp - 1078;   // out = Z 2^p
            const uint32_t lane_addr = tmem + b * S::ACC + ((quad * 32u) << 16);
            // eight columns (four members) of the five accumulators per step; the two steps
            // are unrolled so that their recombinations overlap (28 qubits: 3.40 -> 3.47
            // TB/s; unrolling the transform's member loop too measured slower)
#pragma unroll
            for (uint32_t c0 = part * 16u; c0 < part * 16u + 16u; c0 += 8) {
                float d[5][8];
                tmem_ld8x5(lane_addr + c0, KD, d);
                const uint32_t m0 = c0 >> 1;
                const uint32_t hoff = gbase ^ (((m0 >> 2) & 1u) ? tb[2] : 0u) ^ (((m0 >> 3) & 1u) ? tb[3] : 0u);
                double2 o[4];
#pragma unroll
                for (uint32_t c = 0; c < 4; ++c) {
                    const double re = combine_levels(d[0][2 * c], d[1][2 * c], d[2][2 * c],
                                                     d[3][2 * c], d[4][2 * c], p);
                    const double im = combine_levels(d[0][2 * c + 1], d[1][2 * c + 1], d[2][2 * c + 1],
                                                     d[3][2 * c + 1], d[4][2 * c + 1], p);
                    o[c] = make_double2(re, im);
                }
                if constexpr (XP) xor_unpermute4(o, xl, a.xt, sel_d2);   // o[c] = member c ^ x
#pragma unroll
                for (uint32_t c = 0; c < 4; ++c) out[hoff ^ (XP ? (lo_off[c] ^ cx) : lo_off[c])] = o[c];
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
                        const int32_t row0 = (int32_t)((sl.base(t) + sl.my_off) >> 3);
                        const uint32_t s0 = smem_u32(out + (size_t)lane * seg_amps);
                        for (uint32_t bx = 0; bx < a.boxes; ++bx)
                            tma_store_2d(&a.tmap, 0, row0 + (int32_t)(bx * a.box_rows), s0 + bx * a.box_rows * 128u);
                    } else {
                        bulk_s2g(psi + sl.base(t) + sl.my_off, smem_u32(out + (size_t)lane * seg_amps),
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

sv_status launch_tc64(sv_state *s, const svi::Gate &g0) {
    using S = Tc64;
    using S2 = Tc64S<2>;
    static std::once_flag once;
    static cudaError_t init_err = cudaSuccess;
    std::call_once(once, [] {
        init_err = cudaFuncSetAttribute(apply_tc64<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)S::SMEM);
        if (init_err == cudaSuccess)
            init_err = cudaFuncSetAttribute(apply_tc64<false, 2>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S2::SMEM);
        if (init_err == cudaSuccess)
            init_err = cudaFuncSetAttribute(apply_tc64<false, 1, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    });
    if (init_err != cudaSuccess)
        return svi::set_error(SV_ERR_CUDA, std::string("tensor-core kernel setup: ") +
                                               cudaGetErrorString(init_err));
    svi::Gate gw;
    const svi::Gate *g = &g0;
    if (g0.k < 4) {
        gw = svi::widen_gate(g0, s->n, 4);
        g = &gw;
    }
    Plan p = make_plan(s->n, 4, g->t, S::TB);
    // 16-byte accesses: bank group = tile bits 0..2; the lowest targets there (at most
    // two, the ones inside a group of four members) get a lane-dependent order
    uint32_t tl = 0;
    while (tl < 3u && p.lp[tl] < 3u) ++tl;
    // without the member-order variant and with three or four targets above the low bits
    // (segments of 4 KiB or less), two MMA subtiles per 64 KiB stage: measured at 30
    // qubits, four high targets 11.26 -> 10.58 ms per pass, but two high targets 9.94 ->
    // 10.47 ms, so the mode is kept for the short segments
    // Launches with two targets among the bank bits stage their tiles by tensor-map copies
    // with the 128-byte swizzle instead of taking the XOR member order (one subtile per
    // stage); the others keep 1-D bulk copies, where the swizzled staging measured slower.
    const bool swz = std::min(tl, 2u) >= 2u;
    const bool wide = !swz && s->n >= S2::TB && p.h >= 3;
    if (wide) {
        p = make_plan(s->n, 4, g->t, S2::TB);
        tl = 0;
        while (tl < 3u && p.lp[tl] < 3u) ++tl;
    }
    if (swz) tl = 0;
    Tc64Args a;
    a.box_rows = a.boxes = 0;
    if (swz) {
        const sv_status st = encode_rows_map(s->buf, 16ull << s->n, 16u << p.L, &a.tmap, &a.box_rows, &a.boxes);
        if (st != SV_OK) return st;
    }
    // R (real embedding of U) and its six digits, exactly, on the host
    double rmax = 0.0;
    for (uint32_t i = 0; i < 256; ++i)
        rmax = std::max(rmax, std::max(std::fabs(g->u[i].real()), std::fabs(g->u[i].imag())));
    int eb = 0;
    std::frexp(rmax, &eb);                                   // rmax < 2^eb
    const uint32_t ebias = (uint32_t)std::max(eb + 1022, 1);    // as a biased exponent field
    for (uint32_t n = 0; n < 32; ++n)
        for (uint32_t kk = 0; kk < 32; ++kk) {
            const svi::cplx u = g->u[(n >> 1) * 16 + (kk >> 1)];
            const double r = ((n & 1) == (kk & 1)) ? u.real() : ((n & 1) ? u.imag() : -u.imag());
            int d[6];
            fxp::digits(fxp::to_fixed(fxp::bits_of(r), ebias), d);
            for (int i = 0; i < 6; ++i) a.b[i][n * 32 + kk] = (int16_t)d[i];
        }
    a.b_exp = (int)ebias - 1022;
    a.psi = s->buf;
    a.err = reinterpret_cast<int *>(s->ws + svi::WS_ERR);
    a.ntiles = p.ntiles;
    a.L = p.L;
    a.h = p.h;
    for (int j = 0; j < SV_MAX_K; ++j) a.hi[j] = p.hi[j];
    for (int j = 0; j < 4; ++j) a.lp[j] = p.lp[j];
    a.xs = 3u - tl;
    a.xt = std::min(tl, 2u);
    const unsigned grid = (unsigned)std::min<unsigned long long>(p.ntiles, (unsigned long long)s->num_sms);
    // two targets in bits 0..2 (4-way conflicts and worse) take the swizzled staging; one
    // target there leaves 2-way conflicts, cheaper than either remedy
    if (swz) apply_tc64<false, 1, true><<<grid, S::THREADS, S::SMEM, s->stream>>>(a);
    else if (wide) apply_tc64<false, 2><<<grid, S2::THREADS, S2::SMEM, s->stream>>>(a);
    else apply_tc64<false, 1><<<grid, S::THREADS, S::SMEM, s->stream>>>(a);
    SV_CUDA(cudaGetLastError());
    return SV_OK;
}

}  // namespace svk

namespace svi {

bool tc64_eligible(const sv_state *s, const Gate &g) {
    return s->dtype == SV_C128 && g.k <= 4 && s->n >= svk::Tc64::TB &&
           !(s->policy & SV_POLICY_NO_TENSOR_CORES);
}

sv_status launch_apply_tc64(sv_state *s, const Gate &g) { return svk::launch_tc64(s, g); }

}  // namespace svi
