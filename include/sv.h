/*
 * sv.h -- C ABI of the GB300 state-vector simulator core.
 *
 * The library applies a circuit's gates, after DAG gate fusion has merged runs of gates
 * into dense k-qubit unitaries (k <= 5), to the 2^n complex amplitudes of |psi> on one
 * GPU, and computes the norm, Z-basis probability, Pauli-expectation and top-k
 * reductions.  It follows the paper's statement of the problem:
 *   - a gate is a unitary U_g in C^{2^q x 2^q} plus a tuple of targets (Section 3);
 *   - the pipeline is |psi_out> = E(R(F(P(C)))) (Eq. 5): F = sv_fuse (Section 5.2,
 *     Algorithm 2), R = the precision choice (Eqs. 11-12 plus runtime norm drift),
 *     E = sv_apply_circuit on the GPU;
 *   - a backend offers initialisation, gate application and measurement (Section 4.1):
 *     sv_alloc / sv_set_basis, sv_apply_circuit / sv_apply_gate, sv_probs / sv_expect /
 *     sv_topk / sv_norm.
 *
 * Conventions
 *   - Qubit t is bit t of the amplitude index (little-endian), as fixed by Eq. 3:
 *     (I_{2^{n-t-1}} (x) U (x) I_{2^t}) puts qubit t at stride 2^t.
 *   - Amplitudes are interleaved (re, im): SV_C64 = two floats (8 bytes per amplitude),
 *     SV_C128 = two doubles (16 bytes per amplitude), Eq. 1 / Section 5.4.
 *   - Gate matrices are 2^k x 2^k, row-major, interleaved (re, im) doubles; local index
 *     bit j of the matrix belongs to targets[j].
 *
 * Errors: every call validates its arguments and returns an sv_status; nothing aborts
 * or throws across the ABI.  sv_last_error() returns the calling thread's last message.
 * GPU work is enqueued on the state's stream; calls that return host values (sv_norm,
 * sv_expect, sv_topk, sv_get_state to host, ...) synchronise that stream.  Device-side
 * bounded waits that give up set an error word that the next synchronising call reports
 * as SV_ERR_TIMEOUT.
 *
 * Threading: a state or circuit may be used by one thread at a time; different states
 * may be driven from different threads (each on its own stream).
 */
#ifndef SV_GB300_H
#define SV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = 1,      /* invalid argument (message in sv_last_error) */
    SV_ERR_OOM = 2,      /* device or host allocation failed */
    SV_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    SV_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    SV_ERR_STATE = 5     /* the operation does not fit the state (e.g. buffer too small) */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

#define SV_MAX_K 5         /* widest gate the kernels apply (fused width k <= 5) */
#define SV_MAX_QUBITS 34   /* 2^34 amplitudes */

typedef struct sv_state sv_state;       /* opaque: a device state vector + workspace */
typedef struct sv_circuit sv_circuit;   /* opaque: a fused schedule, host memory */

/* One gate (Section 3): k targets, distinct, each < n; u = 2^k x 2^k complex matrix,
 * row-major interleaved doubles, local bit j <-> targets[j].  Caller owns u. */
typedef struct {
    uint32_t k;
    uint32_t targets[SV_MAX_K];
    const double *u;
} sv_gate;

/* ------------------------------------------------------------------ gate library */

/* The canonical gate set G of Eq. 4 plus the full-unitary gates the workloads use. */
typedef enum {
    SV_GATE_I = 0, SV_GATE_X, SV_GATE_Y, SV_GATE_Z, SV_GATE_H, SV_GATE_S, SV_GATE_T,
    SV_GATE_RX, SV_GATE_RY, SV_GATE_RZ,           /* R_a(theta) = exp(-i theta A / 2) */
    SV_GATE_CNOT, SV_GATE_CZ, SV_GATE_SWAP, SV_GATE_TOFFOLI,
    SV_GATE_U3,                                   /* U3(theta, phi, lambda), OpenQASM 2 form */
    SV_GATE_SQRTX, SV_GATE_SQRTY, SV_GATE_SQRTW,  /* ((1+i) I + (1-i) P) / 2 */
    SV_GATE_FSIM,                                 /* fSim(theta, phi) */
    SV_GATE_CP,                                   /* diag(1, 1, 1, e^{i phi}) */
    SV_GATE_UNITARY                               /* params = the matrix itself */
} sv_gate_kind;

/* Matrix of a gate of the canonical set (Eq. 4).  params: angles (RX/RY/RZ/CP: 1,
 * U3: 3, FSIM: 2, others: 0); for SV_GATE_UNITARY params is the 2^k x 2^k interleaved
 * matrix and nparams = 2 * 4^k.  dagger != 0 returns the adjoint.  u_out must hold
 * 2 * 4^k doubles (at most 2 * 1024); *k_out receives k.  Host only. */
sv_status sv_gate_matrix(uint32_t kind, const double *params, uint32_t nparams, int dagger,
                         double *u_out, uint32_t *k_out);

/* --------------------------------------------------------------------- states */

/* The backend's initialisation operation (Section 4.1): create an n-qubit state
 * (1 <= n <= SV_MAX_QUBITS) in dtype on the current CUDA device, holding the 2^n
 * amplitudes of Eq. 1, initialised to |0...0>.
 *   dev_buf: caller-owned device buffer of `bytes` bytes (16-byte aligned, at least
 *            2^n * 8 (C64) or 2^n * 16 (C128) bytes), or NULL for a library-owned
 *            buffer of exactly the state's size.  A caller buffer must outlive the state.
 *   stream:  cudaStream_t to enqueue all work on (NULL = the legacy default stream).
 * The library also allocates a small workspace (reduction partials, top-k candidates,
 * the error word).  Returns SV_ERR_OOM if an allocation fails. */
sv_status sv_alloc(uint32_t n, sv_dtype dtype, void *dev_buf, size_t bytes, void *stream,
                   sv_state **out);
sv_status sv_free(sv_state *s);                      /* synchronises, frees owned memory */
sv_status sv_info(const sv_state *s, uint32_t *n, sv_dtype *dtype, void **dev_ptr);

/* |x> (x < 2^n).  Asynchronous. */
sv_status sv_set_basis(sv_state *s, uint64_t x);
/* Change the state's precision (e.g. back to SV_C64 after a promotion).  The contents
 * become |0...0> in the new dtype.  A library-owned buffer is reallocated when it is too
 * small; a caller buffer must already hold 2^n amplitudes of the new dtype (else
 * SV_ERR_STATE). */
sv_status sv_set_dtype(sv_state *s, sv_dtype dtype);
/* Copy 2^n amplitudes in the state's dtype from src (host or device memory).  Host
 * sources are copied synchronously; pinned host memory is fastest. */
sv_status sv_set_state(sv_state *s, const void *src, int src_on_device);
/* Read out |psi> = sum_k alpha_k |k> (Eq. 1): copy the 2^n amplitudes (state's dtype,
 * index order, qubit t = bit t) to dst.  To host: synchronises.  To device:
 * asynchronous. */
sv_status sv_get_state(sv_state *s, void *dst, int dst_on_device);

/* ------------------------------------------------------------------ fusion (F) */

/* DAG-based gate fusion, Section 5.1-5.2 (Eq. 8 DAG, Algorithm 2, Eq. 9 product).
 * Gates fuse along DAG edges while the union of their qubits has at most max_k
 * members and contracting the edge keeps the DAG acyclic; U_fused = U_v . U_u in FP64.
 * A vertex's predecessors are tried narrowest union first (ties by gate index).
 * max_k = 0 returns the gates unfused.  Sweeps repeat in min-id topological order
 * until nothing changes; the result is deterministic.  Fused targets are sorted
 * ascending.  Gates wider than max_k are kept as they are (k <= SV_MAX_K).
 * Copies the matrices; free the result with sv_circuit_free.  Host only. */
sv_status sv_fuse(const sv_gate *gates, size_t ngates, uint32_t n, uint32_t max_k,
                  sv_circuit **out);
/* sv_fuse with flags.  SV_FUSE_COMMUTE: commutation-aware fusion (the paper's fusion does
 * no commutativity analysis; Sections 10-11 name it as future work).  Two gates commute
 * when, on every qubit they share, both are diagonal in that qubit (neither changes its
 * bit; exact test on the FP64 entries).  The DAG keeps, per qubit, the edges from a gate
 * not diagonal on it to every gate on it since the previous such gate and from that gate
 * to the diagonal ones after it; the sweeps also contract, after v's predecessors, the
 * vertices that share a qubit with v, are placed before it and have no path to it
 * (ascending id).  Deterministic.  flags = 0 is sv_fuse.  SV_ERR_ARG for unknown flags. */
#define SV_FUSE_COMMUTE 1u
sv_status sv_fuse_ex(const sv_gate *gates, size_t ngates, uint32_t n, uint32_t max_k, uint32_t flags,
                     sv_circuit **out);
/* Fuse `gates` with the decisions sv_fuse made for `pattern` (the gates must act on the
 * same qubits, gate by gate, as the ones `pattern` was fused from, and for a pattern
 * fused with SV_FUSE_COMMUTE be diagonal on the same qubits; matrices may differ -- a
 * parameter sweep).  Algorithm 2's decisions depend only on the qubit sets, so the
 * result equals sv_fuse(gates, n, max_k) bit for bit, without repeating the DAG search.
 * SV_ERR_ARG if the qubits differ.  Host only. */
sv_status sv_fuse_like(const sv_circuit *pattern, const sv_gate *gates, size_t ngates,
                       sv_circuit **out);
sv_status sv_circuit_free(sv_circuit *c);
/* Number of fused gates and the qubit count the circuit was built for. */
sv_status sv_circuit_size(const sv_circuit *c, size_t *nfused, uint32_t *n);
/* Gate i of the schedule: k, targets (k entries, ascending) and matrix (2 * 4^k
 * doubles; may be NULL to skip). */
sv_status sv_circuit_gate(const sv_circuit *c, size_t i, uint32_t *k, uint32_t *targets,
                          double *u);

/* The passes sv_apply_circuit enqueues for the circuit's schedule on a complex64 state of
 * the circuit's width with these SV_POLICY_* flags (two-gate passes: see
 * sv_apply_circuit).  Pass i applies gate first[i] of the schedule, then gate second[i]
 * when second[i] >= 0, in the same pass.  first and second hold room for `cap` entries
 * (the schedule's gate count always suffices); *npasses gets the pass count.
 * SV_ERR_ARG if cap is too small.  Host only. */
sv_status sv_plan_passes(const sv_circuit *c, uint32_t policy, uint32_t *first, int32_t *second,
                         size_t cap, size_t *npasses);

/* ------------------------------------------------------- precision (R) and apply (E) */

/* A-priori rule of Eqs. 11-12: eps_round = g * 2^n * 1.19e-7; complex64 iff
 * eps_round <= eps_tol.  Host only. */
sv_status sv_choose_dtype(uint32_t n, uint64_t g, double eps_tol, sv_dtype *out,
                          double *eps_round);

typedef struct {
    uint32_t adaptive;          /* 1: runtime c64 -> c128 promotion on norm drift */
    double drift_threshold;     /* promote when |norm - norm_before| > this (1e-6) */
    uint32_t drift_check_every; /* check after every S passes (0: only at the end) */
    uint32_t timing;            /* 1: time the gate passes with CUDA events (synchronises) */
} sv_apply_opts;

typedef struct {
    int32_t dtype_used;         /* sv_dtype that produced the final state */
    uint32_t promotions;        /* 1 if the circuit was replayed in complex128 */
    uint64_t passes;            /* HBM passes enqueued (including a replay); a two-gate
                                   pass counts once */
    double norm_before;         /* FP64 norms when adaptive (else 0); norm_before of a basis
                                   start is exactly 1 and takes no pass */
    double norm_after;
    double drift;               /* |norm_after - norm_before| of the reported run */
    uint64_t bytes;             /* algorithmic HBM bytes of the passes: 2 * 2^n * s per dense
                                   pass, 2 * s per touched amplitude of a structured one */
    double apply_ms;            /* with opts->timing: CUDA-event time of all passes (ms) */
    uint64_t tc_passes;         /* passes that ran on the tensor-core kernels */
    uint32_t max_k_used;        /* widest gate of the schedule that produced the final state */
    uint64_t paired_passes;     /* passes that applied two fused gates (SV_POLICY_TWO_GATE_PASSES) */
} sv_apply_report;

/* Apply every gate of the fused schedule, in order, one pass over the state each (Eq. 10:
 * the fused product equals the unfused one).  opts may be NULL (no adaptivity).
 *
 * Two-gate passes (opt-in, SV_POLICY_TWO_GATE_PASSES; complex64 with tensor cores
 * allowed, states of at least 13 qubits): two dense gates of the schedule whose targets,
 * with the low index bits, fit one tile of 2^12 amplitudes (index bits [0, L) plus their
 * targets at or above L, L >= 5) are applied in one read-write pass of the state, the
 * tile kept in shared memory between them.  The second gate of a pair may be taken from
 * further on in the schedule when every gate it passes over acts on other qubits (such
 * gates commute with it; Eq. 8's DAG has no path between them), so the product is the
 * schedule's.  report->passes counts the HBM passes, report->paired_passes those that
 * applied two gates.  A two-gate pass is bound by instruction issue, not HBM: on GB300 it
 * takes 1.8-2.2x the time of a one-gate pass when the tile is contiguous and more when
 * it is gathered from short segments, so it is off by default.
 *
 * Precision (Section 5.4).  complex64 states compute in FP32 (tensor-core passes on exact
 * 9-bit fixed-point slices with FP32-level error relative to each group's largest
 * amplitude).  complex128 states compute to FP64 accuracy: the CUDA-core kernels in FP64
 * FMA; the complex128 tensor-core kernel (gates of up to 4 qubits) in block fixed point,
 * each group of amplitudes on the grid of its largest exponent, with an absolute error
 * per output of at most 2^-46 x (the group's largest amplitude) x (the gate's largest
 * entry) plus half an ulp -- components far below their group's largest keep that
 * absolute accuracy, not FP64's relative one.  A complex128 state runs a circuit that
 * has width-5 gates as the same input gates fused at width 4 (built once per circuit),
 * so that every dense pass stays on the tensor cores (report->max_k_used says which).
 *
 * With opts->adaptive and a C64 state, the FP64 norm is measured before and after (and
 * every drift_check_every passes); if the drift exceeds drift_threshold the state is
 * re-initialised in complex128 from its value at the start of the call and the whole
 * circuit is replayed in complex128 (Section 5.4 made runtime).  A start state that is
 * not a basis state (sv_set_state, or earlier gates) is kept in a complex64 snapshot of
 * 2^n * 8 bytes, allocated on first need and kept by the state until sv_free.
 * Promotion needs a buffer of 2^n * 16 bytes: a library-owned buffer is reallocated (the
 * new one before the old one is released; if memory is short the old one is released
 * first, and if even that fails the call returns SV_ERR_OOM and the state has no buffer:
 * every call but sv_set_dtype, sv_info and sv_free then returns SV_ERR_STATE); a caller
 * buffer must already be that large (else SV_ERR_STATE).  report may be NULL.
 * Asynchronous unless adaptive. */
sv_status sv_apply_circuit(sv_state *s, const sv_circuit *c, const sv_apply_opts *opts,
                           sv_apply_report *report);

/* Apply one gate (unfused per-gate form; targets in any order).  Asynchronous. */
sv_status sv_apply_gate(sv_state *s, const sv_gate *g);

/* ------------------------------------------------------------------ reductions */

/* sum_k |alpha_k|^2 accumulated in FP64 (Eq. 1).  Synchronises. */
sv_status sv_norm(sv_state *s, double *out);
/* The Z-basis measurement distribution of Eq. 1 (the backend's measurement operation,
 * Section 4.1): p_k = |alpha_k|^2 for all 2^n outcomes in index order: float (C64) or
 * double (C128).
 * out_on_device: out is device memory (asynchronous) or host memory (synchronises).  Host
 * memory that is page-locked and mapped for the device (cudaHostAlloc, torch pin_memory)
 * is written by the kernel directly; other host memory goes through a device temporary of
 * the same size. */
sv_status sv_probs(sv_state *s, void *out, int out_on_device);
/* out = sum_t coef[t] <psi| P_t |psi> for Pauli strings P_t given by xmask[t] (X or Y
 * on those qubits) and zmask[t] (Z or Y): P|k> = i^{|x&z|} (-1)^{|k&z|} |k^x>.
 * Accumulated in FP64.  Synchronises. */
sv_status sv_expect(sv_state *s, const uint64_t *xmask, const uint64_t *zmask,
                    const double *coef, size_t nterms, double *out);
/* Noisy simulation with density matrices (Section 9.5): rho on n <= 17 qubits is the
 * 2n-qubit vector v[r + 2^n c] = rho[r, c] (row bits low, column bits high), a state of
 * width 2n made with sv_alloc(2n, ...) and started with sv_set_basis(s, 0) = |0..0><0..0|.
 * sv_fuse_density builds, for every gate U on T, the pair U on T (rows) and conj(U) on
 * T + n (columns), then for each target q the single-qubit depolarizing channel
 * rho -> (1 - p) rho + (p/3)(X rho X + Y rho Y + Z rho Z) as a 4 x 4 matrix on the bits
 * (q, q + n); and fuses the list on 2n qubits by Algorithm 2 (max_k as in sv_fuse).  The
 * result is applied with sv_apply_circuit (adaptive precision does not apply: the norm of
 * v is not conserved).  0 <= p <= 1; n in 1..17. */
sv_status sv_fuse_density(const sv_gate *gates, size_t ngates, uint32_t n, double p, uint32_t max_k,
                          sv_circuit **out);
/* p(x) = Re rho[x, x] for x < 2^(width/2) of a vectorised density matrix (even width):
 * float (C64) or double (C128); host or device memory as in sv_probs. */
sv_status sv_density_probs(sv_state *s, void *out, int out_on_device);
/* Measurement sampling, the backend's third operation (Section 4.1; the paper prints no
 * procedure): nshots outcome indices drawn from p_k = |alpha_k|^2 / sum_j |alpha_j|^2,
 * reproducible bit for bit from an exact integer distribution: P_k = floor(p_k 2^58) with
 * p_k = |alpha_k|^2 in the state's precision; C_k = P_0 + ... + P_k, T = C_{N-1}; shot i:
 * u = SplitMix64(seed + (i+1) * 0x9E3779B97F4A7C15) >> 11 (53 bits), target =
 * floor(u T / 2^53); the outcome is the k with C_{k-1} <= target < C_k.  Outcomes with
 * P_k = 0 are never drawn.  Valid for states of norm below 64 (the sums stay below 2^64).
 * out: nshots uint64 (host or device memory per out_on_device).  Scratch device memory:
 * 2^n / 4 bytes (plus 8 bytes per shot for host output), kept by the state for the next
 * call and released by sv_free.  SV_ERR_STATE if T = 0 (a zero state).  Synchronises. */
sv_status sv_sample(sv_state *s, uint64_t seed, size_t nshots, uint64_t *out, int out_on_device);
/* The min(k, 2^n) most probable outcomes of the Z-basis distribution p_k = |alpha_k|^2
 * (Eq. 1; the backend's measurement operation of Section 4.1 reduced to its head),
 * sorted by probability descending, ties to the lower index.  idx/p are host arrays of
 * k entries.  Synchronises. */
sv_status sv_topk(sv_state *s, uint32_t k, uint64_t *idx, double *p);

/* ------------------------------------------------------ structure-aware application */

/* The paper densifies every fused gate and names the structure it leaves unused among
 * its limits and future work (Sections 10-11).  A gate's structure, exact on its FP64
 * entries (no tolerance):
 *   - local bit j is a CONTROL when U never changes bit j and U is the identity on the
 *     half where bit j is 0;
 *   - V = U restricted to "every control bit is 1", on the other targets, is
 *     SV_STRUCT_DIAGONAL (off-diagonal entries all 0), SV_STRUCT_MONOMIAL (one nonzero in
 *     every row and column: a permutation with phases) or SV_STRUCT_DENSE; a 1 x 1 V equal
 *     to 1 is SV_STRUCT_IDENTITY (U = I).
 * Every pass (sv_apply_gate, sv_apply_circuit) takes this structure into account unless
 * SV_POLICY_DENSE_ONLY is set: amplitudes with a control bit 0 are neither read nor
 * written, diagonal and monomial remainders cost one complex product per amplitude
 * (none where the entry is exactly 1), and the identity launches nothing. */
#define SV_STRUCT_DENSE 0u
#define SV_STRUCT_DIAGONAL 1u
#define SV_STRUCT_MONOMIAL 2u
#define SV_STRUCT_IDENTITY 3u
/* *kind = SV_STRUCT_* of V; *control_mask bit j set when targets[j] is a control (the
 * caller's target order).  Either output may be NULL.  Host only. */
sv_status sv_gate_structure(const sv_gate *g, uint32_t *kind, uint32_t *control_mask);

/* Kernel selection flags for one state (default 0 = automatic: complex64 gates of width
 * 4 and 5 on states of at least k + 7 qubits, and of any width on states of at least 13
 * qubits, run on the tensor cores, complex128 gates of width <= 4 on states of at least 11
 * qubits too, structured gates on the structure-aware kernels, everything else on the CUDA
 * cores). */
#define SV_POLICY_NO_TENSOR_CORES 1u   /* always use the CUDA-core kernels */
#define SV_POLICY_DENSE_ONLY 2u        /* ignore gate structure: every gate a dense pass */
/* sv_probs into page-locked host memory goes through a device buffer of the probabilities'
 * size (2^n * 4 or 8 bytes, allocated on first use and kept by the state until sv_free) and
 * one copy-engine transfer, instead of the kernel writing over the CPU-GPU link itself: the
 * transfer then occupies no SM, so passes of states on other streams run meanwhile. */
#define SV_POLICY_STAGED_PROBS 4u
/* Apply pairs of dense complex64 gates that fit one tile in one pass (two-gate passes; see
 * sv_apply_circuit).  Off by default. */
#define SV_POLICY_TWO_GATE_PASSES 8u
sv_status sv_set_policy(sv_state *s, uint32_t flags);

/* ------------------------------------------------------------ batched execution */

/* A batch: `count` states of n qubits in one dtype, stored back to back (state i at
 * amplitude offset i * 2^n), each driven by its own circuit.  All circuits applied in one
 * call must share their fused structure (same number of fused gates, same targets gate
 * by gate) -- one parameterised circuit family fused with one width; the matrices may
 * differ.  The library keeps a device table of the per-state matrices, processes the
 * states in L2-sized chunks (all gates of a chunk before the next chunk) and captures
 * the launch sequence in a CUDA graph, replayed while the structure and chunking stay
 * the same.  Work is enqueued on the batch's stream. */
typedef struct sv_batch sv_batch;

typedef struct {
    uint32_t chunk_states;   /* states per chunk (0: as many as fit l2_bytes) */
    size_t l2_bytes;         /* chunk budget in bytes (0: 64 MiB) */
    uint32_t no_graph;       /* 1: launch directly instead of through the CUDA graph */
    uint32_t timing;         /* 1: time the passes with CUDA events (synchronises) */
    uint32_t no_tensor_cores; /* 1: complex64 width-4/5 gates on the CUDA cores too (default:
                                 on the tensor cores when n >= 12) */
    uint32_t tile_bits;      /* CUDA-core passes: tiles of 2^tile_bits amplitudes per CTA,
                                10..13 (0: 12 for complex64, 11 for complex128) */
} sv_batch_opts;

typedef struct {
    uint64_t passes;         /* fused gates x states */
    uint64_t launches;       /* kernel launches (fused gates x chunks) */
    uint64_t bytes;          /* algorithmic bytes: passes * 2 * 2^n * s */
    uint32_t chunk_states;
    uint32_t graph_reused;   /* 1 if a previously captured graph was replayed */
    double apply_ms;         /* with opts->timing */
    uint32_t tile_bits;      /* tile size of the CUDA-core passes */
} sv_batch_report;

typedef struct {
    uint32_t best_k;         /* fusion width with the shortest batched apply */
    size_t l2_bytes;         /* chunk budget that achieved it */
    double best_ms;
    double ms[SV_MAX_K + 1]; /* best time per width (index k), 0 if not tried */
    uint32_t cached;         /* 1 if the answer came from the cache */
    uint32_t tile_bits;      /* tile size of the CUDA-core passes (0: the default) */
} sv_tune_result;

/* count in 1..65535; dev_buf: caller buffer of >= count * 2^n * s bytes or NULL.  All
 * states start as |0...0>. */
sv_status sv_batch_alloc(uint32_t n, sv_dtype dtype, uint32_t count, void *dev_buf, size_t bytes,
                         void *stream, sv_batch **out);
sv_status sv_batch_free(sv_batch *b);
sv_status sv_batch_set_basis(sv_batch *b, uint64_t x);     /* every state to |x>; async */
/* Copy state i (2^n amplitudes) to host (synchronises) or device memory. */
sv_status sv_batch_get_state(sv_batch *b, uint32_t i, void *dst, int dst_on_device);
/* Apply circuits[i] to state i for all i < count (see above).  opts and rep may be NULL.
 * SV_ERR_ARG if a circuit does not share the structure of circuits[0]. */
sv_status sv_batch_apply(sv_batch *b, const sv_circuit *const *circuits, const sv_batch_opts *opts,
                         sv_batch_report *rep);
/* out[i] = sum_t coef[t] <psi_i| P_t |psi_i> for every state (host array of count
 * doubles), FP64 accumulation.  Synchronises. */
sv_status sv_batch_expect(sv_batch *b, const uint64_t *xmask, const uint64_t *zmask,
                          const double *coef, size_t nterms, double *out);
sv_status sv_batch_sync(sv_batch *b);
/* Autotuner: fuse `gates` (one representative circuit of the family) at every width
 * kmin..kmax, time the batched apply on this batch for three chunk budgets (64 MiB,
 * 512 MiB, the whole batch) and, when the schedule has CUDA-core passes, for every tile
 * size 10..13 at the width's best chunking; return the fastest (width, chunk budget, tile
 * size).  Results are cached per batch shape and target sequence (the
 * measure-once-and-cache idea of Algorithm 1, applied to the fusion width, the chunking
 * and the tile shape).  Overwrites the batch's states with |0...0>.  Synchronises. */
sv_status sv_batch_tune(sv_batch *b, const sv_gate *gates, size_t ngates, uint32_t kmin, uint32_t kmax,
                        sv_tune_result *out);

/* ------------------------------------------------------------------ serving */

/* A continuous-batching request server on the current device.  Submitted circuits are
 * fused on host threads (Algorithm 2), then admitted -- the least estimated GPU work first
 * (passes x state bytes at the measured pass rates), with aging (a quarter second of work
 * per second waited) so that large requests are not starved -- while their memory
 * (Eq. 14: 2^n s + (2^k)^2 s + workspace) fits the budget and a slot is free; requests
 * that do not fit wait in the queue (no CPU fallback).  Each slot is a pair of CUDA
 * streams (short requests on the high-priority one); the
 * request's state is allocated from the stream-ordered pool, set to |0...0>, every fused
 * pass is applied and the top-k outcomes are returned.  Requests in different slots
 * overlap on the GPU; each result is computed by the same kernels in the same order as
 * alone, so it does not depend on the other requests in flight. */
typedef struct sv_server sv_server;

typedef struct {
    size_t budget_bytes;     /* HBM budget of admitted requests (0: 150 GiB) */
    uint32_t max_slots;      /* requests in flight on the GPU (0: 16; at most 256) */
    uint32_t topk;           /* outcomes per result, 1..64 (0: 64) */
    uint32_t max_k;          /* fusion width 1..5 (0: 5); complex128 requests of 11 or more
                                qubits are fused at min(max_k, 4), the widest gate of the
                                complex128 tensor-core pass */
    uint32_t fuse_threads;   /* host threads that fuse submitted circuits (0: 4) */
} sv_server_config;

typedef struct {
    uint64_t id;             /* as returned by sv_server_submit */
    int32_t status;          /* sv_status of this request */
    int32_t dtype_used;
    uint32_t n;
    uint32_t k;              /* outcomes in idx / p: min(topk, 2^n) */
    uint64_t passes;         /* fused gates applied */
    uint64_t idx[64];        /* most probable outcomes, probability descending, ties to */
    double p[64];            /* the lower index */
    double t_submit, t_admit, t_done;   /* seconds on the server's clock */
} sv_server_result;

typedef struct {
    uint64_t submitted, completed, queued;
    uint32_t active;
    size_t in_use_bytes, budget_bytes;
    double now;              /* the server's clock (seconds since creation) */
} sv_server_stats;

sv_status sv_server_create(const sv_server_config *cfg, sv_server **out);   /* cfg may be NULL */
/* Queue a circuit (gates as for sv_fuse; copied) for an n-qubit state in dtype.  Returns
 * at once with the request id; the latency clock starts here. */
sv_status sv_server_submit(sv_server *s, uint32_t n, sv_dtype dtype, const sv_gate *gates,
                           size_t ngates, uint64_t *id);
/* Move up to cap finished results into out (*nout of them); waits up to wait_ms for the
 * first one when none is ready. */
sv_status sv_server_poll(sv_server *s, sv_server_result *out, size_t cap, size_t *nout, int wait_ms);
sv_status sv_server_get_stats(sv_server *s, sv_server_stats *out);
/* Finish every queued and running request, then release everything. */
sv_status sv_server_destroy(sv_server *s);

/* sum_t coef[t] <psi| P_t |psi> (as sv_expect) for a caller-owned device state, written
 * to out_dev (one double in device memory), enqueued on `stream` (NULL = the legacy
 * default stream) -- without allocating anything.  No counterpart in the paper: it
 * exists for callers that cannot call cudaMalloc or cudaFree, such as a host framework
 * that owns the whole device-memory budget through its own pool, or a latency-critical
 * loop where an allocation would synchronise the device and stall other streams.
 *   psi: 2^n amplitudes in dtype, 16-byte aligned device memory of the current device;
 *        n in 1..34.
 *   out_dev: 8-byte aligned device memory of the current device.  A host pointer or
 *        another device's memory for either is rejected with SV_ERR_ARG.
 * Scratch: a fixed 128 KiB device array inside the library (one FP64 partial per block
 * for each batch of up to 32 terms sharing an X-part; at most 64 batches, else
 * SV_ERR_ARG).  Every GPU that loads the library holds it until the process exits.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the one array, so
 * calls whose work overlaps on the GPU (different streams, no ordering) race; calls on
 * one stream are ordered.  Every scratch slot a call reads is written earlier in the same
 * call, so stale contents from a previous call are never used.  Asynchronous. */
sv_status sv_expect_noalloc(const void *psi, uint32_t n, sv_dtype dtype, const uint64_t *xmask,
                            const uint64_t *zmask, const double *coef, size_t nterms,
                            double *out_dev, void *stream);

/* --------------------------------------------------- global-qubit sharding (2^g GPUs) */

/* The paper keeps the state on one device and names device memory as the design's
 * ceiling (Section 10) and multi-device partitioning as future work (Section 11).  A
 * sharded state splits the 2^n amplitudes by their top g index bits over 2^g processes:
 * rank r holds, as an ordinary state of L = n - g qubits (sv_alloc(L, ...)), the
 * amplitudes r 2^L .. (r + 1) 2^L - 1 in index order.  A plan turns a fused circuit into
 * steps that every rank runs in the same order:
 *   SV_SHARD_APPLY: sv_apply_circuit(shard, segment) -- the gates whose targets are all
 *     local, relabelled to the bit positions their qubits occupy at that point;
 *   SV_SHARD_SWAP (local_bit p, global_bit j): an exchange with the partner rank
 *     r ^ 2^j.  With b = bit j of r, each rank sends the 2^(L-1) amplitudes whose local
 *     index bit p is 1 - b (in index order, e.g. via sv_shard_pack) and puts the
 *     partner's 2^(L-1) amplitudes into the same places (sv_shard_unpack); the qubit at
 *     position p and the one at global position j trade places.
 * Swaps are chosen before each gate that touches a qubit at a global position: the local
 * position whose qubit is used again latest is given up (ties: the highest position,
 * whose half is contiguous).  At the end every qubit is moved back to its own position
 * (exchanges, then SWAP passes inside the shards), so the shards again hold the amplitudes
 * in index order; a norm or a Pauli expectation without X/Y on the top g qubits is then
 * the sum over ranks of the shard's value, with the coefficient's sign from the Z part on
 * the top qubits, (-1)^popcount(zmask >> L & r) (a term with X/Y on top qubits is summed
 * after the same kind of exchange has swapped those qubits into local positions the
 * term does not flip, and swapped back after).  complex128 plans use the circuit's
 * width-4 schedule when it has width-5 gates.  Host only; the transport (NCCL, or a copy
 * between processes) is the caller's. */
#define SV_SHARD_APPLY 0u
#define SV_SHARD_SWAP 1u
typedef struct sv_shard_plan sv_shard_plan;
/* g in 0..16, g < n; SV_ERR_ARG if L = n - g is smaller than the widest gate (or 2). */
sv_status sv_shard_plan_create(const sv_circuit *c, uint32_t g, sv_dtype dtype, sv_shard_plan **out);
sv_status sv_shard_plan_free(sv_shard_plan *p);
/* Steps, exchanges and SWAP passes of the plan. */
sv_status sv_shard_plan_info(const sv_shard_plan *p, size_t *nsteps, uint64_t *exchanges,
                             uint64_t *local_swaps);
/* Step i: its kind, the swap's positions (SV_SHARD_SWAP) or the segment (SV_SHARD_APPLY; a
 * circuit on L qubits owned by the plan, valid until sv_shard_plan_free). */
sv_status sv_shard_plan_step(const sv_shard_plan *p, size_t i, uint32_t *kind, uint32_t *local_bit,
                             uint32_t *global_bit, const sv_circuit **segment);
/* Copy elements offset .. offset + count - 1 of the half of the state whose index bit `bit`
 * is `value` (2^(n-1) amplitudes in index order) to the device buffer dst_dev (pack), or
 * from src_dev back into those places (unpack).  Buffers hold count amplitudes of the
 * state's dtype, 16-byte aligned for complex128 (8-byte for complex64).  Asynchronous on
 * the state's stream; HBM-bound copies. */
sv_status sv_shard_pack(sv_state *s, uint32_t bit, uint32_t value, uint64_t offset, uint64_t count,
                        void *dst_dev);
sv_status sv_shard_unpack(sv_state *s, uint32_t bit, uint32_t value, uint64_t offset, uint64_t count,
                          const void *src_dev);
/* All amplitudes zero (a shard that holds none of |x>).  Asynchronous. */
sv_status sv_set_zero(sv_state *s);

/* Testing aid (no counterpart in the paper): the next `count` allocations of a state
 * buffer (sv_alloc, sv_set_dtype, a promotion) fail as if device memory were exhausted,
 * so that tests can drive the out-of-memory paths without exhausting the GPU.  0 turns
 * it off.  Host only; process-wide. */
sv_status sv_debug_fail_allocs(uint32_t count);

sv_status sv_sync(sv_state *s);   /* wait for the state's stream; reports device errors */
const char *sv_last_error(void);  /* thread-local, never NULL */

#ifdef __cplusplus
}
#endif
#endif /* SV_GB300_H */
