// Measurement sampling, the backend's third operation next to initialisation and gate
// application (Section 4.1).  The paper prints no procedure; this one fixes the order of
// every floating-point step, so the sampled indices are reproducible bit for bit:
//
// 1. p_k = |alpha_k|^2 in the state's precision, widened to FP64.
// 2. Blocks of B = min(64, 2^n) outcomes: S_b = sum of the block's p_k in index order.
// 3. Chunks of C = min(4096, #blocks) blocks: L_b = exclusive prefix of the S_b within the
//    chunk (index order), chunk totals, O_c = exclusive prefix of the totals (index order),
//    T = their sum; the block prefix is P_b = O_{chunk(b)} + L_b.
// 4. Shot i: u = (SplitMix64(seed + (i + 1) * 0x9E3779B97F4A7C15) >> 11) * 2^-53 (Steele,
//    Lea and Flood's generator as an output function of a counter), target = u * T.
// 5. b = the largest block with P_b <= target and S_b > 0; r = target - P_b; the outcome is
//    the block's first k whose running sum exceeds r, else its last outcome with p_k > 0.
//
// Step 2 reads the state once (one thread per block, FP64 adds: about 4 ms at 30 qubits,
// bound by this GPU's FP64 rate); steps 3-4 touch 2^n / 64 doubles; each shot reads one
// block of the state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "sv_internal.h"

namespace svk {

constexpr unsigned long long SM_GAMMA = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// |alpha|^2 in the state's precision, no contraction, widened to FP64.
__device__ __forceinline__ double sprob(const float2 *psi, unsigned long long k) {
    const float2 v = psi[k];
    return (double)__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
}
__device__ __forceinline__ double sprob(const double2 *psi, unsigned long long k) {
    const double2 v = psi[k];
    return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
}

template <typename C>
__global__ void block_sums(const C *__restrict__ psi, unsigned long long nb, uint32_t B,
                           double *__restrict__ S) {
    for (unsigned long long b = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; b < nb;
         b += (unsigned long long)gridDim.x * blockDim.x) {
        double c = 0.0;
        for (uint32_t j = 0; j < B; ++j) c = __dadd_rn(c, sprob(psi, b * B + j));
        S[b] = c;
    }
}

__global__ void chunk_scan(const double *__restrict__ S, unsigned long long nc, uint32_t C,
                           double *__restrict__ L, double *__restrict__ tot) {
    for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < nc;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (uint32_t j = 0; j < C; ++j) {
            L[c * C + j] = acc;
            acc = __dadd_rn(acc, S[c * C + j]);
        }
        tot[c] = acc;
    }
}

// one thread: O_c and T (written at O[nc])
__global__ void chunk_offsets(const double *__restrict__ tot, unsigned long long nc, double *O) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double acc = 0.0;
    for (unsigned long long c = 0; c < nc; ++c) {
        O[c] = acc;
        acc = __dadd_rn(acc, tot[c]);
    }
    O[nc] = acc;
}

template <typename C>
__global__ void draw_shots(const C *__restrict__ psi, const double *__restrict__ S,
                           const double *__restrict__ L, const double *__restrict__ O,
                           unsigned long long nb, uint32_t B, uint32_t Cb, unsigned long long nc,
                           unsigned long long seed, unsigned long long nshots,
                           unsigned long long *__restrict__ out) {
    const double T = O[nc];
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         i < nshots; i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long z = splitmix64(seed + (i + 1) * SM_GAMMA);
        const double u = __dmul_rn(__ull2double_rn(z >> 11), 0x1p-53);   // exact
        const double target = __dmul_rn(u, T);
        // the largest b with P_b <= target (P_0 = 0 <= target)
        unsigned long long lo = 0, hi = nb - 1;
        while (lo < hi) {
            const unsigned long long mid = lo + (hi - lo + 1) / 2;
            const double P = __dadd_rn(O[mid / Cb], L[mid]);
            if (P <= target) lo = mid;
            else hi = mid - 1;
        }
        unsigned long long b = lo;
        while (S[b] == 0.0 && b > 0) --b;        // the first block with S_b > 0 has P_b = 0
        const double r = __dsub_rn(target, __dadd_rn(O[b / Cb], L[b]));
        double c = 0.0;
        long long k = -1, last_nz = -1;
        for (uint32_t j = 0; j < B; ++j) {
            const double p = sprob(psi, b * B + j);
            if (p > 0.0) last_nz = j;
            c = __dadd_rn(c, p);
            if (c > r) {
                k = j;
                break;
            }
        }
        if (k < 0) {
            // running sum never exceeded r (rounding at the block's end): its last outcome
            // with p > 0
            for (uint32_t j = B; j-- > 0;)
                if (sprob(psi, b * B + j) > 0.0) { last_nz = j; break; }
            k = last_nz < 0 ? (long long)B - 1 : last_nz;
        }
        out[i] = b * B + (unsigned long long)k;
    }
}

}  // namespace svk

using namespace svi;

extern "C" sv_status sv_sample(sv_state *s, uint64_t seed, size_t nshots, uint64_t *out,
                               int out_on_device) {
    clear_error();
    if (!s || !out) return set_error(SV_ERR_ARG, "sv_sample: null argument");
    if (nshots == 0) return SV_OK;
    const unsigned long long N = 1ull << s->n;
    const uint32_t B = (uint32_t)std::min<unsigned long long>(64, N);
    const unsigned long long nb = N / B;
    const uint32_t Cb = (uint32_t)std::min<unsigned long long>(4096, nb);
    const unsigned long long nc = nb / Cb;
    double *S = nullptr, *L = nullptr, *tot = nullptr, *O = nullptr;
    unsigned long long *dout = nullptr;
    cudaStream_t st = s->stream;
    SV_CUDA(cudaMallocAsync(&S, nb * sizeof(double), st));
    sv_status rc = SV_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        if (rc == SV_OK && e != cudaSuccess)
            rc = set_error(e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA,
                           std::string("sv_sample: ") + what + ": " + cudaGetErrorString(e));
    };
    fail(cudaMallocAsync(&L, nb * sizeof(double), st), "alloc");
    fail(cudaMallocAsync(&tot, nc * sizeof(double), st), "alloc");
    fail(cudaMallocAsync(&O, (nc + 1) * sizeof(double), st), "alloc");
    if (!out_on_device) fail(cudaMallocAsync(&dout, nshots * sizeof(unsigned long long), st), "alloc");
    if (rc == SV_OK) {
        const int grid = s->num_sms * 8;
        if (s->dtype == SV_C64)
            svk::block_sums<<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(s->buf), nb, B, S);
        else
            svk::block_sums<<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(s->buf), nb, B, S);
        fail(cudaGetLastError(), "block sums");
        svk::chunk_scan<<<(unsigned)std::min<unsigned long long>((nc + 127) / 128, 65535), 128, 0, st>>>(
            S, nc, Cb, L, tot);
        fail(cudaGetLastError(), "chunk scan");
        svk::chunk_offsets<<<1, 32, 0, st>>>(tot, nc, O);
        fail(cudaGetLastError(), "chunk offsets");
    }
    double T = 0.0;
    if (rc == SV_OK) {
        fail(cudaMemcpyAsync(&T, O + nc, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
        fail(cudaStreamSynchronize(st), "sync");
        if (rc == SV_OK && !(T > 0.0)) rc = set_error(SV_ERR_STATE, "sv_sample: the state has zero norm");
    }
    if (rc == SV_OK) {
        unsigned long long *dst = out_on_device ? reinterpret_cast<unsigned long long *>(out) : dout;
        const unsigned grid = (unsigned)std::min<unsigned long long>((nshots + 255) / 256,
                                                                     (unsigned long long)s->num_sms * 32);
        if (s->dtype == SV_C64)
            svk::draw_shots<<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(s->buf), S, L, O, nb,
                                                  B, Cb, nc, seed, nshots, dst);
        else
            svk::draw_shots<<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(s->buf), S, L, O, nb,
                                                  B, Cb, nc, seed, nshots, dst);
        fail(cudaGetLastError(), "shots");
        if (!out_on_device && rc == SV_OK)
            fail(cudaMemcpyAsync(out, dout, nshots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
                 "copy");
    }
    cudaFreeAsync(S, st);
    if (L) cudaFreeAsync(L, st);
    if (tot) cudaFreeAsync(tot, st);
    if (O) cudaFreeAsync(O, st);
    if (dout) cudaFreeAsync(dout, st);
    if (rc != SV_OK) return rc;
    if (!out_on_device) return check_device_error(s);
    return SV_OK;
}
