/*
 * sv.h -- C ABI of libsv, a GB300 (sm_103a) state-vector simulator for the
 * data-parallel path of the JUQCS method (Willsch et al., "Benchmarking
 * Supercomputers with the Juelich Universal Quantum Computer Simulator",
 * arXiv:1912.03243).
 *
 * Conventions shared by every call
 * --------------------------------
 * State.  An n-qubit state is 2^n complex amplitudes (Sec. 2, after Eq. 1).
 *   Qubit j is bit j of the amplitude index (qubit 0 = least significant);
 *   the paper leaves the order open.  Storage by dtype:
 *     SV_C64    2^n x {float re, float im}, interleaved, 8 B per amplitude.
 *     SV_C128   2^n x {double re, double im}, 16 B per amplitude: the exact
 *               ("JUQCS-E") representation of Sec. 1, 2^(n+4) bytes.
 *     SV_ENC2B  the adaptive two-byte code of Sec. 1 ("JUQCS-A"): 2^n x
 *               {int8 re, int8 im} codes followed by 2^(n-8) float block
 *               scales (one per 256 consecutive amplitudes; one scale when
 *               n < 8).  Amplitude x = sign(q) * scale * fl(|q|/127).
 *   sv_bytes_required() gives the exact device footprint of each layout.
 * Matrices.  Complex matrices are row-major, each entry (re, im) as two
 *   doubles.  A 2x2 gate is 8 doubles: u00 u01 u10 u11.
 * Ownership.  Handles belong to the library until sv_free().  Every array a
 *   caller passes (matrices, qubit lists, indices, outputs, circuit text) is
 *   caller-owned, read or written only during the call, never retained.
 *   A buffer given to sv_attach stays owned by the caller and must outlive
 *   the handle.
 * Streams.  Each handle is bound to one CUDA stream (NULL = the legacy
 *   default stream).  Gate calls only enqueue work and return; kernel faults
 *   surface as SV_ERR_CUDA at the next call that synchronises (sv_sync,
 *   sv_norm, sv_amplitudes, sv_copy_to_host, sv_get_codes).
 * Errors.  Every call returns an sv_status; nothing is thrown across the ABI.
 *   On failure the state is unchanged when the failure is an argument
 *   check (checked before any launch) and undefined after SV_ERR_CUDA.
 *   sv_last_error() returns a thread-local message for the last failure.
 * Sizes.  1 <= n <= 40 for SV_C64/SV_C128 and 1 <= n <= 40 for SV_ENC2B,
 *   further limited by free device memory (checked before allocating).
 * Fault injection (host side, for tests): while the environment variable
 *   SV_FAULT_INJECT=alloc|launch|sync is set, every allocation, launch or
 *   synchronisation reports SV_ERR_OOM / SV_ERR_CUDA without touching the
 *   GPU; SV_FAULT_INJECT=tc_wait makes the tensor-core kernel skip its MMA
 *   so that its bounded wait runs out (SV_ERR_TIMEOUT at the next
 *   synchronising call, the context stays usable).
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_state *sv_handle;
typedef struct sv_plan_s *sv_plan;
typedef struct sv_batch_s *sv_batch;

typedef enum { SV_C64 = 0, SV_C128 = 1, SV_ENC2B = 2 } sv_dtype;

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = 1,          /* bad argument (range, repeated qubit, NULL) */
    SV_ERR_OOM = 2,          /* not enough free device memory */
    SV_ERR_DTYPE = 3,        /* operation not defined for this dtype */
    SV_ERR_CUDA = 4,         /* a CUDA call or kernel failed */
    SV_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    SV_ERR_STATE = 6,        /* handle in the wrong state (freed, busy) */
    SV_ERR_PARSE = 7,        /* circuit text could not be parsed */
    SV_ERR_UNSUPPORTED = 8   /* valid request outside what is implemented */
} sv_status;

/* Circuit execution modes (sv_run_circuit, sv_plan_create). */
typedef enum {
    SV_MODE_PERGATE = 0,     /* one HBM pass per gate (Eq. 1 per gate) */
    SV_MODE_TILED = 1,       /* many gates per HBM pass: 2^13-amplitude tiles in
                                shared memory, one compiled kernel per pass */
    SV_MODE_FUSED = 2,       /* gates fused into dense k-qubit blocks (k = 3..6
                                chosen by the planner), one HBM pass per block on
                                the tensor cores */
    SV_MODE_AUTO = 3         /* measured choice: sv_plan_create plans every
                                candidate (tiled with each register-bit, CTA and
                                HBM-I/O configuration of the generator; fused
                                with k = 3..6; per-gate where no tile fits),
                                times each on a scratch state of the handle's
                                size and keeps the fastest; the choice is
                                remembered per device, n, dtype and circuit
                                (sv_plan_tuning reports it) */
} sv_mode;

/* ---- lifecycle --------------------------------------------------------- */

/* Device bytes an n-qubit state of dtype dt occupies (0 if n is out of
 * range).  SV_C128: 2^(n+4) (Sec. 1). */
size_t sv_bytes_required(int n, sv_dtype dt);

/* Allocate an n-qubit state on the current device with cudaMalloc and set it
 * to |0...0> (Sec. 4: the machine starts in |0>).  stream: a cudaStream_t
 * or NULL.  Errors: SV_ERR_ARG (n, dt, out), SV_ERR_OOM (checked against
 * cudaMemGetInfo before allocating), SV_ERR_CUDA. */
sv_status sv_alloc(int n, sv_dtype dt, void *stream, sv_handle *out);

/* Wrap caller-owned device memory (e.g. a torch tensor) of at least
 * sv_bytes_required(n, dt) bytes, 256-byte aligned.  The contents are left
 * as they are.  Errors: SV_ERR_ARG (NULL, too small, misaligned). */
sv_status sv_attach(int n, sv_dtype dt, void *dev_ptr, size_t bytes, void *stream, sv_handle *out);

/* Synchronise and release the handle (and its memory if sv_alloc made it).
 * NULL is accepted and ignored. */
sv_status sv_free(sv_handle h);

/* Set the state to the computational basis state |idx>.  Errors: SV_ERR_ARG
 * (idx >= 2^n). */
sv_status sv_set_basis(sv_handle h, uint64_t idx);

/* Block until all work queued on the handle's stream is done; report any
 * device fault. */
sv_status sv_sync(sv_handle h);

/* Thread-local message describing the last failure ("" if none). */
const char *sv_last_error(void);

/* Qubit count / dtype of a handle (-1 on a NULL handle). */
int sv_num_qubits(sv_handle h);
int sv_dtype_of(sv_handle h);

/* ---- gates --------------------------------------------------------------- */

/* Eq. 1: for every index pair (i, i + 2^target) with bit `target` clear
 * (and bit `control` set when control >= 0), replace (a_i, a_{i+2^target})
 * by U (a_i, a_{i+2^target}).  U: 8 doubles, 2x2 row-major.  Two-qubit
 * controlled gates of the paper (CNOT of Sec. 3, CZ of Sec. 4) are this
 * call with U = X or Z.  Every dtype: SV_ENC2B decodes each touched block,
 * applies the gate in FP32 and re-encodes (Sec. 3, the "encoding-decoding
 * operation").  Errors: SV_ERR_ARG (target/control out of range or equal,
 * U NULL). */
sv_status sv_apply_gate(sv_handle h, int target, int control, const double *U);

/* Sec. 2: a k-qubit gate as a dense 2^k x 2^k matrix on the listed qubits
 * (local index bit j <-> qubits[j]; qubits[0] is the least significant).
 * 1 <= k <= 6, qubits distinct.  SV_C64 states of n >= 12 apply it on the
 * tensor cores (tcgen05) with split-precision BF16 products (A_hi B_hi +
 * A_hi B_lo + A_lo B_hi) and FP32 accumulation; smaller SV_C64 states in
 * FP32 and SV_C128 in FP64 on the CUDA cores.  The tensor-core kernel's only
 * wait is bounded; if it gives up, the next synchronising call returns
 * SV_ERR_TIMEOUT, after which the state and the CUDA context are undefined
 * (MMAs still in flight may write freed tensor memory) and must be
 * discarded.  Errors: SV_ERR_ARG, SV_ERR_DTYPE (SV_ENC2B). */
sv_status sv_apply_fused(sv_handle h, int k, const int *qubits, const double *U);

/* ---- circuits -------------------------------------------------------------- */

/* Run a circuit given as text (one gate per line: "H 3", "CZ 0 1",
 * "CP 2 5 0.785", "U 4 <8 doubles>", see the package documentation) on the
 * handle's current state, with one of the sv_mode strategies.  All modes
 * compute the same product of gate matrices (Sec. 2); they differ in how
 * many HBM passes they make.  SV_ENC2B supports SV_MODE_PERGATE (and
 * SV_MODE_AUTO, which then has only that candidate).  Errors: SV_ERR_PARSE,
 * SV_ERR_ARG (qubit range), SV_ERR_DTYPE. */
sv_status sv_run_circuit(sv_handle h, const char *text, int mode);

/* Plan a circuit once (parse, classify gates, group them into HBM passes,
 * upload the pass programs) and execute it many times.  The plan is bound
 * to the handle and must be freed before it.  SV_MODE_AUTO times its
 * candidates here, on a scratch state that it cudaMallocs and frees (the
 * handle's state is not touched); without room for one it takes the tiled
 * plan.  Its first tuning of a large circuit takes seconds (every candidate
 * is compiled and run three times). */
sv_status sv_plan_create(sv_handle h, const char *text, int mode, sv_plan *out);
/* Execute a plan on the handle's stream (asynchronous).  The first execution
 * launches the kernels one by one; the second captures them into a CUDA graph
 * on a stream the plan owns, and every later one replays that graph; the
 * plan's stream waits for the handle's stream before the graph and the
 * handle's stream waits for the graph after it, so the order of work on the
 * handle's stream is unchanged.  Plans with CUDA-core dense blocks (host
 * matrix copies per launch), single-launch plans and runs with SV_GRAPH=0
 * always launch directly; so does a plan whose capture failed. */
sv_status sv_plan_execute(sv_plan p);
/* *out = 1 if the plan's executions now replay a CUDA graph, else 0. */
sv_status sv_plan_uses_graph(sv_plan p, int *out);
/* Statistics of a plan: number of gates, HBM passes (kernel launches) and
 * the algorithmic bytes all passes move. */
sv_status sv_plan_info(sv_plan p, int64_t *gates, int64_t *passes, double *bytes);
/* Per-launch timing hook: execute the plan and record event[i] (caller-
 * created cudaEvent_t) before launch i and event[passes] after the last. */
sv_status sv_plan_execute_timed(sv_plan p, void *const *events, int64_t n_events);
/* The autotuner's record of an SV_MODE_AUTO plan as JSON text: each
 * candidate strategy with its measured ms per execution and the chosen one
 * ({"timed": false, ...} when the choice was remembered from an earlier
 * tuning, there was one candidate only, or no scratch state fitted); "" for
 * other modes.  buf (cap bytes,
 * NUL-terminated, may be NULL), *len = the full length. */
sv_status sv_plan_tuning(sv_plan p, char *buf, size_t cap, size_t *len);
sv_status sv_plan_free(sv_plan p);
/* Launch i of a plan (0 <= i < passes): the name of the kernel it runs and
 * the algorithmic bytes it moves.  *kernel points to a static string. */
sv_status sv_plan_launch_info(sv_plan p, int64_t i, const char **kernel, double *bytes);

/* Launch i of a plan: for a compiled tile pass, the FP32 lane operations per
 * amplitude its gates need at least (2 per structured butterfly such as H,
 * SX, SY; 1 per T-type phase; 4 per other complex phase; 8 per dense 2x2;
 * times the fraction of amplitudes its controls leave; sign flips and X
 * free) and its register segments (shared-memory transpositions + 1); 0 and
 * 0 for other launches.  Either pointer may be NULL. */
sv_status sv_plan_launch_stats(sv_plan p, int64_t i, double *fp32_ops_per_amplitude, int64_t *segments);

/* Host only (no GPU needed): the generated CUDA source of pass `pass` of the
 * SV_MODE_TILED plan of a circuit (what a plan compiles with NVRTC), into
 * buf (cap bytes, NUL-terminated, truncated if short; buf may be NULL);
 * *len receives the full length.  Errors: SV_ERR_PARSE, SV_ERR_ARG (pass out
 * of range), SV_ERR_UNSUPPORTED (n below one tile). */
sv_status sv_plan_pass_source(const char *text, int n, sv_dtype dt, int64_t pass, char *buf, size_t cap,
                              size_t *len);

/* Host only (no GPU needed): plan a circuit for SV_MODE_TILED and report its
 * gate count, HBM passes and register segments; with compile != 0 also
 * compile every pass for sm_103a (the tiled mode compiles one straight-line
 * kernel per pass with NVRTC when a plan is created).  n >= 13 (SV_C64) or
 * n >= 12 (SV_C128).  Errors: SV_ERR_PARSE, SV_ERR_ARG, SV_ERR_UNSUPPORTED,
 * SV_ERR_CUDA (compile failure). */
sv_status sv_plan_stats(const char *text, int n, sv_dtype dt, int compile, int64_t *gates, int64_t *passes,
                        int64_t *segments);

/* Host only (no GPU needed): which tensor-core kernel a dense k-qubit block
 * on these qubits of an n-qubit complex64 state runs (Sec. 2: the block acts
 * on the amplitudes that differ only in its qubits; the library's kernel for
 * it is chosen from the qubit layout) and, when it loads its tiles with
 * tensor-map copies, the map's layout: the tile's 12 qubits (tile_pos, bit t
 * of a tile index is state qubit tile_pos[t]); tma_rank dimensions, where
 * dimension d holds the qubits from tma_start[d] up to the next start (the
 * last up to n), of size dim[d], byte stride stride[d - 1] for d >= 1 (8-byte
 * elements), box[d] elements copied; tma_nbox boxes per tile at global
 * element offsets tma_boff[b] from the tile's base, laid out one after the
 * other in shared memory.  Without tensor-map loads tma_rank = tma_nbox = 0
 * and the map fields are 0.  kernel (cap bytes, NUL-terminated, may be NULL)
 * receives the launch name (k_fused_tc<k=..>, k_fused_tc<k=..,tma> or
 * k_fused_tc_groups<k=..>); every other output may be NULL (arrays: 12, 5,
 * 4, 5, 4 and 5 entries).  Errors: SV_ERR_ARG (n outside 12..40, k outside
 * 1..6, repeated or out-of-range qubits). */
sv_status sv_fused_tc_layout(int n, int k, const int *qubits, char *kernel, size_t cap, int *tile_pos,
                             int *tma_rank, int *tma_nbox, int *tma_start, uint64_t *tma_boff, uint64_t *dim,
                             uint64_t *stride, uint32_t *box);

/* ---- batches of independent circuits ------------------------------------------ */

/* A batch of count independent circuits, member k = texts[k] on its own
 * state handles[k] (SV_C64 or SV_C128, sizes may differ, no state shared,
 * all on one device).  Each member is planned as in SV_MODE_TILED (per-gate
 * updates below one tile).  sv_batch_execute runs all members together: on
 * its first call with direct launches, then as one CUDA graph in which each
 * member is an independent chain of its launches, so passes of different
 * members run concurrently and small states no longer leave the GPU idle
 * (Sec. 4: independent terms; the same holds for unrelated circuits).  The
 * batch runs on a private stream that every member handle's stream is
 * joined to by events before and after, so work queued on them stays in
 * order (sv_batch_execute is asynchronous like a gate call).  Ownership: the batch holds one plan per member (the handles must
 * outlive it; free the batch first).  Errors: SV_ERR_ARG (NULL, count < 1 or
 * > 4096, a state shared by two members, mixed devices), SV_ERR_DTYPE
 * (SV_ENC2B), SV_ERR_PARSE, plus those of sv_plan_create. */
sv_status sv_batch_create(const sv_handle *handles, const char *const *texts, int count, sv_batch *out);
/* Run every member's circuit once on its current state (asynchronous). */
sv_status sv_batch_execute(sv_batch b);
/* Gates of all members, their launches per execution, algorithmic bytes,
 * and whether executions now replay the graph (any pointer may be NULL). */
sv_status sv_batch_info(sv_batch b, int64_t *gates, int64_t *launches, double *bytes, int *uses_graph);
sv_status sv_batch_free(sv_batch b);
/* Create, execute once and free. */
sv_status sv_run_batch(const sv_handle *handles, const char *const *texts, int count);

/* ---- two-byte encoding (Sec. 1 and Sec. 3) ---------------------------------- */

/* Encode an SV_C64 state into an SV_ENC2B state of the same n (blocks of 256,
 * scale = max(|re|,|im|), q = rint(x * fl(127/scale)) clamped to +-127).
 * Errors: SV_ERR_DTYPE, SV_ERR_ARG (n differs). */
sv_status sv_encode2b(sv_handle src_c64, sv_handle dst_enc);
/* Decode an SV_ENC2B state into an SV_C64 state. */
sv_status sv_decode2b(sv_handle src_enc, sv_handle dst_c64);
/* Copy the raw codes (2^(n+1) int8) and scales (max(1, 2^(n-8)) float) of an
 * SV_ENC2B state to host memory (either pointer may be NULL). */
sv_status sv_get_codes(sv_handle h, int8_t *codes, float *scales);

/* ---- read-out ---------------------------------------------------------------- */

/* Gather m amplitudes psi[idx[j]] into out[2j], out[2j+1] (host doubles).
 * idx: host array of m indices < 2^n.  Synchronises. */
sv_status sv_amplitudes(sv_handle h, size_t m, const uint64_t *idx, double *out);

/* sum_i |psi_i|^2 in FP64 (partial sums of at most 8 squares in the storage
 * precision, FP64 beyond), deterministic.  Synchronises. */
sv_status sv_norm(sv_handle h, double *out);

/* Expectation values <psi| sigma^alpha_i |psi> for every qubit i and
 * alpha = x, y, z (Sec. 3: the validation observable is
 * <Q_alpha(i)> = (1 - <sigma^alpha_i>)/2 of the normalised state).
 * out: caller-owned host array of 3n doubles, out[3 i + alpha] with
 * alpha 0 = x, 1 = y, 2 = z; not divided by the norm.  Works on SV_C64,
 * SV_C128 and SV_ENC2B (decoded on the fly, codes untouched).  Read-only
 * passes over the state in tiles of 2^13 amplitudes (2^12 for SV_C128):
 * the first holds qubits 0..12, each later one keeps the low qubits (3, or
 * SV_EXPECT_LOW in 3..8; the 8 in-block ones for SV_ENC2B) and takes the
 * next uncovered ones: 1 + ceil((n - 13) / 10) passes for SV_C64.  Sums in
 * the storage precision over a few tiles, FP64 beyond.  Synchronises.
 * Errors: SV_ERR_ARG (NULL), SV_ERR_UNSUPPORTED (more than 40 qubits outside
 * one tile), SV_ERR_OOM (the partial-sum scratch, kept in the handle and
 * grown on first use) or SV_ERR_CUDA. */
sv_status sv_expect_pauli(sv_handle h, double *out);

/* Raw copy of the whole state between device and host memory (bytes must be
 * sv_bytes_required).  Synchronises. */
sv_status sv_copy_to_host(sv_handle h, void *dst, size_t bytes);
sv_status sv_copy_from_host(sv_handle h, const void *src, size_t bytes);

/* Gather m amplitudes from caller-owned device memory without allocating any
 * device memory (the paper has no counterpart; this is a library service).
 * For callers that cannot call cudaMalloc -- an allocator that owns all of
 * HBM, a state that fills the device, a loop that must not hit cudaMalloc's
 * implicit synchronisation -- and so cannot create a handle either (handles
 * hold cudaMalloc'ed scratch).  state: device pointer to an n-qubit state in
 * the dtype layout above; idx: m host indices < 2^n; out: 2m host doubles
 * (re, im).  At most 65536 indices per call (larger m is rejected with
 * SV_ERR_ARG and a message); the index list and results pass through one
 * fixed 1.5 MiB file-scope device array that every GPU loading the library
 * holds until exit.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current, so make the first
 * call before any stream capture.  Every call shares the array: calls that
 * overlap on the GPU (other threads, other streams) race.  Synchronises the
 * stream.  The state pointer is checked on the host before any copy or
 * launch: it must be device memory of the current device
 * (cudaPointerGetAttributes), aligned to 16 bytes for SV_C128 and 8 bytes
 * otherwise, and, where the driver reports the allocation's extent, hold
 * sv_bytes_required(n, dt) bytes from the pointer on; a host pointer, a
 * pointer of another device, a misaligned or too-short buffer is SV_ERR_ARG
 * with a message.  Errors: SV_ERR_ARG, SV_ERR_CUDA. */
sv_status sv_amplitudes_noalloc(const void *state, int n, sv_dtype dt, size_t m, const uint64_t *idx,
                                double *out, void *stream);

/* ---- decomposition of entangling gates (Sec. 4) ---------------------------------- */

/* Eq. 3: <z|C|0> for m bit strings z of an n-qubit circuit C (n <= 64),
 * without the 2^n state.  Qubits in maskA form partition A, the others B.
 * Every CZ/CP between A and B is decomposed (a CX between them is first
 * written as H CZ H); the 2^S terms are simulated as 2^S x 2 half-size
 * complex64 state vectors batched into one launch per pass, and the
 * products of their coefficients are summed in FP64.  form 0: projector
 * decomposition CP = P0 (x) 1 + P1 (x) P(theta); form 1: Eq. 2 (CZ only,
 * weight 1/2 per decomposed gate).  z: host, out: 2m host doubles.
 * n_cut_out (may be NULL) receives S.  stream: cudaStream_t or NULL.
 * Errors: SV_ERR_PARSE, SV_ERR_ARG, SV_ERR_UNSUPPORTED (SWAP across the
 * cut, CP in form 1, S > 16), SV_ERR_OOM. */
sv_status sv_cut_amplitudes(const char *text, int n, uint64_t maskA, int form, size_t m,
                            const uint64_t *z, double *out, int *n_cut_out, void *stream);

/* The part of the Eq. 3 sum over the branches s with s mod 2^nparts_log2 ==
 * part (Sec. 4: the terms are independent, so parts can be computed on
 * different GPUs or processes and added).  The low nparts_log2 branch bits
 * are fixed, which turns their branch operators into plain diagonal gates and
 * halves the batched vectors per fixed bit.  Summing all 2^nparts_log2 parts
 * gives sv_cut_amplitudes.  0 <= nparts_log2 <= 16, part < 2^nparts_log2
 * (parts with no branch give zeros).  Other arguments and errors as
 * sv_cut_amplitudes. */
sv_status sv_cut_amplitudes_part(const char *text, int n, uint64_t maskA, int form, uint64_t part, int nparts_log2,
                                 size_t m, const uint64_t *z, double *out, int *n_cut_out, void *stream);

/* The Eq. 3 sum over the branches of several parts at once: the parts
 * parts[0..nlist-1] of 2^nparts_log2 (each < 2^nparts_log2, none repeated,
 * 1 <= nlist <= 2^nparts_log2), as sv_cut_amplitudes_part would give them
 * one by one, added in FP64 on the device (Sec. 4: the terms are
 * independent, so a process or GPU sums its share and one reduction over
 * them all gives <z|C|0>).  The parts run one after another on the same
 * device buffers, so memory is that of one part.  A rank r of W processes
 * takes nparts_log2 = ceil(log2 W) and the parts p with p mod W = r.  Other
 * arguments and errors as sv_cut_amplitudes_part; SV_ERR_ARG for a bad
 * list. */
sv_status sv_cut_amplitudes_parts(const char *text, int n, uint64_t maskA, int form, int nparts_log2, size_t nlist,
                                  const uint64_t *parts, size_t m, const uint64_t *z, double *out, int *n_cut_out,
                                  void *stream);

/* Eq. 3 over P partitions (Sec. 4: the sum over s of products of P
 * circuits that each act on one partition, with memory bound by the largest
 * partition's dimension).  part_of[q] in 0..P-1 gives the partition of each
 * of the n qubits (2 <= n <= 128, 2 <= P <= 16, every partition nonempty and
 * at most 40 qubits plus its cuts' branch bits).  Every CZ, CP or CX between
 * two partitions is a decomposed gate; each partition holds the branch bits
 * of the cuts that touch it.  z: m bit strings of ceil(n / 64) little-endian
 * 64-bit words each (qubit q is bit q % 64 of word q / 64).  part and
 * nparts_log2 as sv_cut_amplitudes_part (0, 0 for the whole sum).  Other
 * arguments and errors as sv_cut_amplitudes; SV_ERR_UNSUPPORTED also when
 * more than 16 branch bits are batched or a partition is too large. */
sv_status sv_cut_amplitudes_multi(const char *text, int n, const uint8_t *part_of, int P, int form, uint64_t part,
                                  int nparts_log2, size_t m, const uint64_t *z, double *out, int *n_cut_out,
                                  void *stream);

/* sv_cut_amplitudes_parts over P partitions: the listed branch parts of
 * sv_cut_amplitudes_multi summed in FP64 on the device.  Arguments and
 * errors as sv_cut_amplitudes_multi and sv_cut_amplitudes_parts. */
sv_status sv_cut_amplitudes_multi_parts(const char *text, int n, const uint8_t *part_of, int P, int form,
                                        int nparts_log2, size_t nlist, const uint64_t *parts, size_t m,
                                        const uint64_t *z, double *out, int *n_cut_out, void *stream);

/* ---- host-only helpers (no GPU needed) -------------------------------------------- */

/* The library's own matrix for a named gate of the circuit format: writes 8
 * doubles (1-qubit) or 32 doubles (2-qubit, local index = bit(first) +
 * 2 bit(second)); returns 1 or 2 qubits, or -1 if the name is unknown. */
int sv_gate_matrix(const char *name, const double *params, int n_params, double *out);

/* Library version string. */
const char *sv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SV_H */
