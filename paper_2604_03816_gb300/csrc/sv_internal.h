// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "sv.h"

namespace svi {

using cplx = std::complex<double>;

// Thread-local last error message; set() returns the status for `return svi::set(...)`.
sv_status set_error(sv_status st, const std::string &msg);
void clear_error();

// A gate on sorted targets with its FP64 matrix (row-major, 2^k x 2^k).
struct Gate {
    uint32_t k = 0;
    uint32_t t[SV_MAX_K] = {0, 0, 0, 0, 0};
    std::vector<cplx> u;
};

// Relabel a gate's local bits so that its targets are ascending (same operator).
Gate sorted_gate(uint32_t k, const uint32_t *targets, const double *u);

// Exact structure of a sorted gate (structure.cpp): its control qubits and the reduced
// gate V on the other targets (U = I except where every control bit is 1, V there).
struct Structure {
    uint32_t kind = SV_STRUCT_DENSE;   // of V: SV_STRUCT_*
    uint32_t ctrl = 0;                 // local control bits of the gate
    uint32_t nctrl = 0;
    uint32_t ctrl_q[SV_MAX_K] = {0, 0, 0, 0, 0};   // their qubits, ascending
    Gate v;                            // reduced gate (k = 0 for a 1 x 1 V)
};
Structure classify(const Gate &g);

// The decisions of one run of Algorithm 2: contractions (u absorbs v) in order and the
// final topological order of the surviving vertices.
struct FusePlan {
    std::vector<std::pair<int, int>> contractions;
    std::vector<int> order;
};

// Algorithm 2 over sorted gates (fuse.cpp); records its decisions in *plan if given;
// commute: the commutation-aware DAG and contractions of commuting vertices.
std::vector<Gate> fuse_gates(const std::vector<Gate> &in, uint32_t n, uint32_t max_k,
                             FusePlan *plan = nullptr, bool commute = false);
// Bit j set when the gate never changes its local bit j (fuse.cpp).
uint32_t diagonal_mask(const Gate &g);
// g as an m-qubit gate U (x) I (m >= g.k, m <= n; fuse.cpp).
Gate widen_gate(const Gate &g, uint32_t n, uint32_t m);
// g as an m-qubit gate U (x) I on the sorted qubits qs (containing g's targets).
Gate widen_gate_on(const Gate &g, const uint32_t *qs, uint32_t m);
// Apply a recorded plan to gates with the same qubit sets (fuse.cpp).
std::vector<Gate> replay_fusion(std::vector<Gate> nodes, const FusePlan &plan);

}  // namespace svi

struct sv_circuit {
    uint32_t n = 0;
    std::vector<svi::Gate> gates;
    // the input gates (targets sorted), kept so that complex128 states can run the same
    // circuit fused at the tensor-core kernel's widest width (4) instead of applying
    // width-5 gates on the FP64 CUDA cores; that schedule is built on first use
    std::vector<svi::Gate> in_gates;
    mutable std::once_flag narrow_once;
    mutable std::vector<svi::Gate> narrow;
    // how it was fused, for sv_fuse_like: input qubit sets and the recorded plan
    uint32_t max_k = 0;
    uint32_t flags = 0;               // SV_FUSE_* it was fused with
    std::vector<uint32_t> in_k;
    std::vector<uint32_t> in_t;       // SV_MAX_K per input gate, sorted
    std::vector<uint32_t> in_diag;    // with SV_FUSE_COMMUTE: diagonal_mask of each input gate
    svi::FusePlan plan;
};

// Device workspace layout (bytes), carved from one allocation.
namespace svi {
constexpr size_t WS_ERR = 0;                   // int error word (+ padding)
constexpr size_t WS_PARTIAL = 256;             // double partials[WS_NPARTIAL]
constexpr int WS_NPARTIAL = 8192;
constexpr size_t WS_RESULT = WS_PARTIAL + WS_NPARTIAL * 8;   // double results[64]
constexpr size_t WS_TOPK = WS_RESULT + 64 * 8;               // top-k candidates
constexpr int TOPK_MAX_WARPS = 4096;
constexpr size_t WS_TOPK_BYTES = size_t(TOPK_MAX_WARPS) * 64 * 16;
constexpr size_t WS_BYTES = WS_TOPK + WS_TOPK_BYTES + 64 * 16;
}  // namespace svi

struct sv_state {
    uint32_t n = 0;
    sv_dtype dtype = SV_C64;
    void *buf = nullptr;        // amplitudes
    size_t cap = 0;             // bytes available at buf
    bool owned = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    unsigned char *ws = nullptr;   // device workspace (WS_BYTES)
    // what the state holds, for adaptive replay: a basis state or a snapshot
    bool basis_known = true;
    uint64_t basis_x = 0;
    void *snap = nullptr;       // library-owned snapshot of the initial state (c64)
    size_t snap_cap = 0;
    int num_sms = 0;
    uint32_t policy = 0;        // SV_POLICY_* flags (kernel selection)
    void *samp = nullptr;       // sampling scratch (sample.cu), kept across calls
    size_t samp_cap = 0;
    void *probs_buf = nullptr;  // SV_POLICY_STAGED_PROBS: device probabilities, kept across calls
    size_t probs_cap = 0;
};

namespace svi {
// Which kernel family ran a pass (launch_apply's optional out-parameter).
enum PassKind { PASS_CUDA_CORE = 0, PASS_TENSOR_CORE = 1, PASS_STRUCTURED = 2 };
}  // namespace svi

// One batched launch: gate k/t applied to `states` consecutive states at psi with
// per-state matrices at utab (batch.cu).
struct sv_batch_launch {
    sv_dtype dtype = SV_C64;
    uint32_t k = 0, n = 0;
    uint32_t t[SV_MAX_K] = {0, 0, 0, 0, 0};
    uint32_t states = 0;
    void *psi = nullptr;
    const void *utab = nullptr;
    int *err = nullptr;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    bool tc = false;            // complex64 width 4/5 on the tensor cores (apply_tc.cu)
    uint32_t tile_bits = 0;     // CUDA-core passes: 2^tile_bits amplitudes per CTA (0: default)
};

namespace svk {
cudaError_t tc_batch_prepare();
sv_status launch_tc_batch(const sv_batch_launch &L);
// `bytes` bytes at buf as a 2-D tensor of 128-byte rows for TMA tensor copies with the
// 128-byte shared-memory swizzle; a segment of seg_bytes is *boxes boxes of *box_rows rows
// (apply_tc.cu).  `map` points to a CUtensorMap.
sv_status encode_rows_map(void *buf, unsigned long long bytes, uint32_t seg_bytes, struct CUtensorMap_st *map,
                          uint32_t *box_rows, uint32_t *boxes);
}  // namespace svk

namespace svi {
// ---- kernels (apply_kernels.cu / reduce_kernels.cu); all enqueue on s->stream ----
// One pass of g; *bytes (if given) gets the pass's algorithmic HBM bytes: a full read and
// write of the state, or of the amplitudes a structure-aware pass touches.
sv_status launch_apply(sv_state *s, const Gate &g, uint64_t *bytes = nullptr, int *kind = nullptr);
// Structure-aware pass (apply_struct.cu): is it preferred over the dense kernels, and run it.
bool struct_preferred(const sv_state *s, const Structure &st);
sv_status launch_apply_struct(sv_state *s, const Structure &st, uint64_t *bytes);
bool tc_eligible(const sv_state *s, const Gate &g);        // apply_tc.cu
sv_status launch_apply_tc(sv_state *s, const Gate &g);
bool tc64_eligible(const sv_state *s, const Gate &g);      // apply_tc64.cu
sv_status launch_apply_tc64(sv_state *s, const Gate &g);
// Two complex64 gates in one pass (apply_tc2.cu): do they fit one tile, and run them
// (g0 first).
bool tc2_pair_fits(const sv_state *s, const Gate &g0, const Gate &g1);
sv_status launch_apply_tc2(sv_state *s, const Gate &g0, const Gate &g1);
sv_status launch_norm(sv_state *s, double *dev_out);     // writes one double on device
sv_status launch_probs(sv_state *s, void *dev_out);
sv_status launch_density_probs(sv_state *s, void *dev_out);   // Re v[x + 2^(n/2) x]
sv_status launch_expect(sv_state *s, const uint64_t *x, const uint64_t *z, const double *c,
                        size_t nterms, double *host_out);
sv_status launch_topk(sv_state *s, uint32_t k, uint64_t *idx, double *p);
sv_status enqueue_topk(sv_state *s, double *host_p, unsigned long long *host_i);
sv_status launch_widen(sv_state *s, const void *src_c64, void *dst_c128);
sv_status launch_set_one(sv_state *s, uint64_t x);
sv_status check_device_error(sv_state *s);   // synchronises; reads and clears the error word
// The circuit's input gates fused again at width <= 4 when its schedule has width-5 gates
// (built once per circuit), else its schedule: what complex128 runs on the tensor cores.
const std::vector<Gate> &narrow_schedule(const sv_circuit *c);
// SV_ERR_STATE (with a message) when a failed reallocation left the state without a buffer.
sv_status check_live(const sv_state *s, const char *who);
sv_status enqueue_expect_sum(const void *psi, uint32_t n, sv_dtype dtype, const uint64_t *x,
                             const uint64_t *z, const double *c, size_t nterms, double *scratch,
                             size_t scratch_doubles, int nb_fixed, double *out_dev,
                             cudaStream_t stream);
}  // namespace svi

#define SV_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return svi::set_error(e_ == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA, \
                                  std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)
