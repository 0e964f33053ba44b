// Inline-PTX helpers for sm_103a: mbarrier, 1-D bulk (TMA) copies between global and
// shared memory, proxy fences and a bounded wait.  Every wait here gives up after a
// deadline measured on %globaltimer and reports failure instead of spinning forever.
#pragma once

#include <cstdint>

namespace svk {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity to complete; false after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_test_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// Plain arrive (count 1) on an mbarrier; release semantics at CTA scope.
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Potentially blocking test (no suspend-time hint): the thread may be suspended until the
// phase completes or a hardware time limit passes, instead of polling shared memory.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for a phase, giving up when *abort is set by another role or after limit_ns (then
// setting *abort).  Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity,
                                                   volatile int *abort,
                                                   uint64_t limit_ns = 2000000000ull) {
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (globaltimer_ns() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// Named barrier over `count` threads with an AND-reduction of `pred` (uniform result).
__device__ __forceinline__ bool named_bar_and(uint32_t id, uint32_t count, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.and.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void named_bar(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Wait until at most N committed bulk-store groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Global -> shared bulk copy (TMA, non-tensor); completion counted on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst_smem, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst_smem), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Shared -> global bulk copy, tracked by the issuing thread's bulk groups.
__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 ::"l"(dst), "r"(src_smem), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until all committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Wait until all committed bulk stores have completed.
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Make this thread's generic-proxy shared-memory accesses visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Global -> shared copy of one box of a 2-D tensor map (tile mode) at coordinates (x, y);
// completion counted on the mbarrier.  x times the element size must be a multiple of 16
// bytes; the tensor map lives in kernel parameter space (__grid_constant__).
__device__ __forceinline__ void tma_load_2d(uint32_t dst_smem, const void *tmap, int32_t x, int32_t y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst_smem), "l"(tmap), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared -> global copy of one box of a 2-D tensor map at (x, y), tracked by the issuing
// thread's bulk groups.  x, y >= 0.
__device__ __forceinline__ void tma_store_2d(const void *tmap, int32_t x, int32_t y, uint32_t src_smem) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(tmap), "r"(x), "r"(y), "r"(src_smem)
                 : "memory");
}

// The 128-byte swizzle of TMA tensor copies, for 8-byte elements at index f of a
// 1024-byte-aligned shared-memory tile: the 16-byte chunk (index bits 1-3) is XORed with
// the 128-byte row within the 1024-byte block (index bits 4-6).  It is linear over XOR, so
// swz(a ^ b) = swz(a) ^ swz(b), and its own inverse.
__device__ __forceinline__ uint32_t swz128(uint32_t f) {
    return f ^ ((f >> 3) & 0xEu);
}

// Tile addressing for the warp that moves a tile: lane i (< 2^h) owns segment i of every
// tile, whose offset from the tile's base it computes once; the tile base deposits the
// tile index around the h high target bits.  The high-target positions live in
// registers, so no per-segment constant-bank loads remain on the copy path.
struct SegLanes {
    uint32_t L, h;
    uint32_t hi[5];
    unsigned long long my_off;   // this lane's segment offset (amplitudes)

    __device__ __forceinline__ void init(uint32_t L_, uint32_t h_, const uint32_t *hi_, uint32_t lane) {
        L = L_;
        h = h_;
        my_off = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            hi[j] = j < (int)h ? hi_[j] : 0u;
            if (j < (int)h && ((lane >> j) & 1u)) my_off |= 1ull << hi[j];
        }
    }
    __device__ __forceinline__ unsigned long long base(unsigned long long t) const {
        unsigned long long b = t << L;
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if (j < (int)h) {
                const unsigned long long lo = b & ((1ull << hi[j]) - 1ull);
                b = ((b >> hi[j]) << (hi[j] + 1)) | lo;
            }
        return b;
    }
};

// Insert a zero bit at position p of x (bits >= p move up by one).
__device__ __forceinline__ uint64_t insert_zero64(uint64_t x, uint32_t p) {
    const uint64_t lo = x & ((1ull << p) - 1ull);
    return ((x >> p) << (p + 1)) | lo;
}
__device__ __forceinline__ uint32_t insert_zero32(uint32_t x, uint32_t p) {
    const uint32_t lo = x & ((1u << p) - 1u);
    return ((x >> p) << (p + 1)) | lo;
}

}  // namespace svk
