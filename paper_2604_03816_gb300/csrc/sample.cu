// Measurement sampling, the backend's third operation next to initialisation and gate
// application (Section 4.1).  The paper prints no procedure; this one draws from an exact
// integer cumulative distribution, so the sampled indices are reproducible bit for bit
// and every prefix sum may be formed in parallel:
//
// 1. p_k = |alpha_k|^2 in the state's precision (FP32 for complex64, FP64 for
//    complex128), no contraction.
// 2. P_k = floor(p_k 2^58), from the bits of p_k (exponent and mantissa, integer shifts).
// 3. Blocks of B = min(64, 2^n) outcomes: S_b = sum of the block's P_k (uint64, one warp
//    per block); chunks of C = min(4096, #blocks) blocks: L_b = exclusive prefix of the
//    S_b within the chunk (a shared-memory scan), chunk totals, O_c = their exclusive
//    prefix and T = the total; the block prefix is P_b = O_{chunk(b)} + L_b.
// 4. Shot i: z = SplitMix64(seed + (i + 1) * 0x9E3779B97F4A7C15) (Steele, Lea and Flood's
//    generator as an output function of a counter), target = floor((z >> 11) T / 2^53),
//    one 64 x 64 -> 128-bit high product.
// 5. b = the largest block with P_b <= target (then target < P_b + S_b: S_b > 0); the
//    outcome is the block's first k whose running sum of P exceeds target - P_b.
//
// Step 3 reads the state once (coalesced, integer work only for complex64; complex128
// computes p_k on the FP64 pipe); each shot reads one block of the state.  The scratch
// arrays stay allocated in the state between calls (2^n / 4 bytes plus the shots).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "sv_internal.h"

namespace svk {

constexpr unsigned long long SM_GAMMA = 0x9E3779B97F4A7C15ull;
constexpr int SCALE_BITS = 58;
constexpr uint32_t SCAN_THREADS = 512, SCAN_ITEMS = 8;   // chunk = 4096 blocks

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// floor(p 2^58) from the IEEE bits of p >= 0.
__device__ __forceinline__ unsigned long long fixed_of(float p) {
    const uint32_t b = __float_as_uint(p);
    const int e = (int)(b >> 23);
    if (e == 0) return 0ull;                                  // below 2^-126: floor is 0
    const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u; // p = m 2^(e - 150)
    const int sh = e - 150 + SCALE_BITS;
    if (sh >= 0) return m << sh;
    return sh <= -64 ? 0ull : m >> (-sh);
}
__device__ __forceinline__ unsigned long long fixed_of(double p) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(p);
    const int e = (int)(b >> 52);
    if (e == 0) return 0ull;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // p = m 2^(e - 1075)
    const int sh = e - 1075 + SCALE_BITS;
    if (sh >= 0) return m << sh;
    return sh <= -64 ? 0ull : m >> (-sh);
}

// P_k of amplitude k: |alpha|^2 in the state's precision, no contraction.
__device__ __forceinline__ unsigned long long pfix(const float2 *psi, unsigned long long k) {
    const float2 v = psi[k];
    return fixed_of(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
}
__device__ __forceinline__ unsigned long long pfix(const double2 *psi, unsigned long long k) {
    const double2 v = psi[k];
    return fixed_of(__dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)));
}

// P of the two adjacent amplitudes 2j, 2j + 1 (one 16-byte load for complex64).
__device__ __forceinline__ unsigned long long pfix2(const float2 *psi, unsigned long long j) {
    const float4 v = reinterpret_cast<const float4 *>(psi)[j];
    return fixed_of(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y))) +
           fixed_of(__fadd_rn(__fmul_rn(v.z, v.z), __fmul_rn(v.w, v.w)));
}
__device__ __forceinline__ unsigned long long pfix2(const double2 *psi, unsigned long long j) {
    return pfix(psi, 2 * j) + pfix(psi, 2 * j + 1);
}

// One warp per block of B = 64 outcomes (two adjacent ones per lane), four blocks in
// flight per warp; B < 64 (n < 6): one block, lane l takes outcomes l and l + 32.
template <typename C>
__global__ void block_sums(const C *__restrict__ psi, unsigned long long nb, uint32_t B,
                           unsigned long long *__restrict__ S) {
    constexpr int ILP = 4;
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned long long wid = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    if (B < 64) {
        if (wid == 0) {
            unsigned long long s = 0;
            if (lane < B) s = pfix(psi, lane);
            if (lane + 32 < B) s += pfix(psi, lane + 32);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) S[0] = s;
        }
        return;
    }
    for (unsigned long long b0 = wid; b0 < nb; b0 += ILP * nw) {
        unsigned long long s[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const unsigned long long b = b0 + (unsigned long long)u * nw;
            s[u] = b < nb ? pfix2(psi, b * 32 + lane) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
            const unsigned long long b = b0 + (unsigned long long)u * nw;
            if (lane == 0 && b < nb) S[b] = s[u];
        }
    }
}

// Chunk c of C = SCAN_THREADS x SCAN_ITEMS blocks (or all nb < C): exclusive prefix L of
// its S and its total tot[c], by a shared-memory scan (the sums are exact integers, so
// the order does not matter).
__global__ void __launch_bounds__(SCAN_THREADS) chunk_scan(const unsigned long long *__restrict__ S,
                                                           unsigned long long nb, uint32_t C,
                                                           unsigned long long *__restrict__ L,
                                                           unsigned long long *__restrict__ tot) {
    __shared__ unsigned long long part[SCAN_THREADS];
    const unsigned long long c = blockIdx.x;
    const unsigned long long base = c * C;
    const uint32_t t = threadIdx.x;
    unsigned long long v[SCAN_ITEMS];
    unsigned long long s = 0;
#pragma unroll
    for (uint32_t i = 0; i < SCAN_ITEMS; ++i) {
        const unsigned long long j = base + (unsigned long long)t * SCAN_ITEMS + i;
        v[i] = (t * SCAN_ITEMS + i < C && j < nb) ? S[j] : 0ull;
        s += v[i];
    }
    part[t] = s;
    __syncthreads();
    for (uint32_t o = 1; o < SCAN_THREADS; o <<= 1) {          // inclusive Hillis-Steele
        const unsigned long long add = t >= o ? part[t - o] : 0ull;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    unsigned long long run = t ? part[t - 1] : 0ull;            // exclusive
#pragma unroll
    for (uint32_t i = 0; i < SCAN_ITEMS; ++i) {
        const unsigned long long j = base + (unsigned long long)t * SCAN_ITEMS + i;
        if (t * SCAN_ITEMS + i < C && j < nb) L[j] = run;
        run += v[i];
    }
    if (t == SCAN_THREADS - 1) tot[c] = part[t];
}

// One block: O_c = exclusive prefix of the chunk totals, and T at O[nc].
__global__ void __launch_bounds__(1024) chunk_offsets(const unsigned long long *__restrict__ tot,
                                                      unsigned long long nc,
                                                      unsigned long long *__restrict__ O) {
    __shared__ unsigned long long part[1024];
    __shared__ unsigned long long carry;
    const uint32_t t = threadIdx.x;
    if (t == 0) carry = 0;
    __syncthreads();
    for (unsigned long long c0 = 0; c0 < nc; c0 += 1024) {
        const unsigned long long j = c0 + t;
        const unsigned long long x = j < nc ? tot[j] : 0ull;
        part[t] = x;
        __syncthreads();
        for (uint32_t o = 1; o < 1024; o <<= 1) {
            const unsigned long long add = t >= o ? part[t - o] : 0ull;
            __syncthreads();
            part[t] += add;
            __syncthreads();
        }
        if (j < nc) O[j] = carry + part[t] - x;
        __syncthreads();
        if (t == 0) carry += part[1023];
        __syncthreads();
    }
    if (t == 0) O[nc] = carry;
}

template <typename C>
__global__ void draw_shots(const C *__restrict__ psi, const unsigned long long *__restrict__ L,
                           const unsigned long long *__restrict__ O, unsigned long long nb, uint32_t B,
                           uint32_t Cb, unsigned long long nc, unsigned long long seed,
                           unsigned long long nshots, unsigned long long *__restrict__ out) {
    const unsigned long long T = O[nc];
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         i < nshots; i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long z = splitmix64(seed + (i + 1) * SM_GAMMA);
        const unsigned long long target = __umul64hi((z >> 11) << 11, T);   // floor(u53 T / 2^53)
        // the largest b with P_b <= target (P_0 = 0 <= target)
        unsigned long long lo = 0, hi = nb - 1;
        while (lo < hi) {
            const unsigned long long mid = lo + (hi - lo + 1) / 2;
            if (O[mid / Cb] + L[mid] <= target) lo = mid;
            else hi = mid - 1;
        }
        const unsigned long long b = lo;
        const unsigned long long r = target - (O[b / Cb] + L[b]);   // < S_b
        unsigned long long c = 0;
        uint32_t k = B - 1;
        for (uint32_t j = 0; j < B; ++j) {
            c += pfix(psi, b * B + j);
            if (c > r) {
                k = j;
                break;
            }
        }
        out[i] = b * B + k;
    }
}

}  // namespace svk

using namespace svi;

extern "C" sv_status sv_sample(sv_state *s, uint64_t seed, size_t nshots, uint64_t *out,
                               int out_on_device) {
    clear_error();
    if (!s || !out) return set_error(SV_ERR_ARG, "sv_sample: null argument");
    if (check_live(s, "sv_sample") != SV_OK) return SV_ERR_STATE;
    if (nshots == 0) return SV_OK;
    const unsigned long long N = 1ull << s->n;
    const uint32_t B = (uint32_t)std::min<unsigned long long>(64, N);
    const unsigned long long nb = N / B;
    const uint32_t Cb = (uint32_t)std::min<unsigned long long>(svk::SCAN_THREADS * svk::SCAN_ITEMS, nb);
    const unsigned long long nc = (nb + Cb - 1) / Cb;
    cudaStream_t st = s->stream;
    sv_status rc = SV_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        if (rc == SV_OK && e != cudaSuccess)
            rc = set_error(e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA,
                           std::string("sv_sample: ") + what + ": " + cudaGetErrorString(e));
    };
    // scratch S, L, tot, O (and the shots for host output), kept in the state across calls
    const size_t words = 2 * nb + 2 * nc + 1 + (out_on_device ? 0 : nshots);
    if (s->samp_cap < words * sizeof(unsigned long long)) {
        SV_CUDA(cudaStreamSynchronize(st));
        if (s->samp) cudaFree(s->samp);
        s->samp = nullptr;
        s->samp_cap = 0;
        SV_CUDA(cudaMalloc(&s->samp, words * sizeof(unsigned long long)));
        s->samp_cap = words * sizeof(unsigned long long);
    }
    unsigned long long *S = static_cast<unsigned long long *>(s->samp);
    unsigned long long *L = S + nb, *tot = L + nb, *O = tot + nc;
    unsigned long long *dout = out_on_device ? nullptr : O + nc + 1;
    if (rc == SV_OK) {
        const unsigned grid = (unsigned)std::min<unsigned long long>((nb * 32 + 255) / 256,
                                                                     (unsigned long long)s->num_sms * 16);
        if (s->dtype == SV_C64)
            svk::block_sums<<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(s->buf), nb, B, S);
        else
            svk::block_sums<<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(s->buf), nb, B, S);
        fail(cudaGetLastError(), "block sums");
        svk::chunk_scan<<<(unsigned)nc, svk::SCAN_THREADS, 0, st>>>(S, nb, Cb, L, tot);
        fail(cudaGetLastError(), "chunk scan");
        svk::chunk_offsets<<<1, 1024, 0, st>>>(tot, nc, O);
        fail(cudaGetLastError(), "chunk offsets");
    }
    unsigned long long T = 0;
    if (rc == SV_OK) {
        fail(cudaMemcpyAsync(&T, O + nc, sizeof(T), cudaMemcpyDeviceToHost, st), "copy");
        fail(cudaStreamSynchronize(st), "sync");
        if (rc == SV_OK && T == 0)
            rc = set_error(SV_ERR_STATE, "sv_sample: the state has no probability mass to sample");
    }
    if (rc == SV_OK) {
        unsigned long long *dst = out_on_device ? reinterpret_cast<unsigned long long *>(out) : dout;
        const unsigned grid = (unsigned)std::min<unsigned long long>((nshots + 255) / 256,
                                                                     (unsigned long long)s->num_sms * 32);
        if (s->dtype == SV_C64)
            svk::draw_shots<<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(s->buf), L, O, nb, B,
                                                  Cb, nc, seed, nshots, dst);
        else
            svk::draw_shots<<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(s->buf), L, O, nb, B,
                                                  Cb, nc, seed, nshots, dst);
        fail(cudaGetLastError(), "shots");
        if (!out_on_device && rc == SV_OK)
            fail(cudaMemcpyAsync(out, dout, nshots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
                 "copy");
    }
    if (rc != SV_OK) return rc;
    if (!out_on_device) return check_device_error(s);
    return SV_OK;
}
