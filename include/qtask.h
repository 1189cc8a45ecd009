/*
 * qtask.h -- C ABI of libqtask.so, an incremental state-vector quantum-circuit
 * simulator for one NVIDIA GB300 (sm_103a).
 *
 * Method: qTask (T.-W. Huang, arXiv 2210.01076).  A circuit on n qubits is an
 * ordered list of levels ("nets", Section III-B); the gates of one level act
 * on disjoint qubits.  The simulator keeps the 2^n complex amplitudes
 * (Section II-A; qubit q is bit q of the amplitude index, q_0 least
 * significant, Listing 1) split into fixed partitions of 2^log2_partition
 * consecutive amplitudes (the paper's blocks, Section III-C).  Circuit
 * modifiers (insert/remove/replace a gate, insert/remove a level; Table 2)
 * only record the edit; qt_update_state then re-simulates only the partitions
 * downstream of the edits (Sections III-D and III-E), starting from device
 * checkpoints of the state kept at segment boundaries (the per-net state
 * vectors of Section III-F).  The result is bit-identical to a full
 * re-simulation of the edited circuit (qt_update_state with force_full = 1).
 *
 * Ownership: the library owns every host and device buffer it allocates; the
 * caller owns every buffer it passes in (gates are copied, never retained).
 * Errors: every call returns a qt_status; no C++ exception crosses the ABI.
 * qt_last_error(c) returns a message for the last failed call on c.
 * Threading: calls on different circuits may run concurrently; calls on one
 * circuit must be serialised by the caller.
 * Device: all GPU work of a circuit runs on one CUDA stream (the library's
 * own, or the one given to qt_set_stream).  Device memory is allocated on the
 * first call that needs the GPU (qt_update_state, qt_read_amplitudes*,
 * qt_norm), not by qt_create, so circuit editing works without a GPU.
 */
#ifndef QTASK_H
#define QTASK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qt_circuit qt_circuit;

typedef enum {
    QT_OK = 0,
    QT_ERR_ARG = 1,       /* bad argument (null pointer, bad qubit, bad kind, ...) */
    QT_ERR_CONFLICT = 2,  /* the gate shares a qubit with a gate of its level (Section III-B) */
    QT_ERR_RANGE = 3,     /* level or amplitude index out of range */
    QT_ERR_NOT_FOUND = 4, /* no gate with that id in that level */
    QT_ERR_OOM = 5,       /* device memory (or the mem_limit option) exhausted; nothing changed */
    QT_ERR_CUDA = 6,      /* a CUDA call failed (including: no GPU present) */
    QT_ERR_STALE = 7,     /* edits are pending: call qt_update_state first */
    QT_ERR_TIMEOUT = 8    /* a bounded device wait expired */
} qt_status;

/* Amplitude storage and arithmetic.
 *   QT_C128    16 B per amplitude, IEEE binary64 (re, im); FP64 arithmetic.
 *   QT_C64      8 B per amplitude, binary32 (re, im); FP32 arithmetic.
 *   QT_C128_DF 16 B per amplitude as float-float pairs (re_hi, re_lo, im_hi,
 *              im_lo), each real held as an unevaluated sum of two binary32
 *              values (about 48 significand bits); arithmetic in float-float
 *              on the FP32 pipes, whose rate on GB300 is ~60x its FP64 rate.
 * qt_read_amplitudes returns binary64 (re, im) pairs for QT_C128 and
 * QT_C128_DF, binary32 pairs for QT_C64. */
typedef enum { QT_C128 = 0, QT_C64 = 1, QT_C128_DF = 2 } qt_dtype;

/* Gate kinds: the paper's standard gates (Table 1) and the composites it
 * names (CZ, CCX, SWAP; Section III-A), plus U3 and the controlled phase CP.
 * Matrices (c = cos(t/2), s = sin(t/2), t = theta[0]):
 *   H = [[1,1],[1,-1]]/sqrt2, X = [[0,1],[1,0]], Y = [[0,-i],[i,0]],
 *   Z = diag(1,-1), S = diag(1,i), SDG = diag(1,-i), T = diag(1,e^{i pi/4}),
 *   TDG = diag(1,e^{-i pi/4}), RX = [[c,-is],[-is,c]], RY = [[c,-s],[s,c]],
 *   RZ = diag(e^{-it/2}, e^{it/2}),
 *   U3(t,p,l) = [[c, -e^{il}s], [e^{ip}s, e^{i(p+l)}c]]  (p = theta[1], l = theta[2]),
 *   CNOT = X on target[0] controlled by control[0]; CZ = Z controlled;
 *   CCX = X controlled by control[0] and control[1];
 *   CP = diag(1, e^{i theta[0]}) on target[0] controlled by control[0];
 *   SWAP exchanges target[0] and target[1]. */
typedef enum {
    QT_H = 0, QT_X, QT_Y, QT_Z, QT_S, QT_SDG, QT_T, QT_TDG, QT_RX, QT_RY, QT_RZ, QT_U3,
    QT_CNOT, QT_CZ, QT_SWAP, QT_CCX, QT_CP, QT_NUM_KINDS
} qt_kind;

/* A gate.  ntarget/ncontrol must match the kind (1/0 for one-qubit gates,
 * 1/1 for CNOT CZ CP, 2/0 for SWAP, 1/2 for CCX); all qubits distinct and
 * in [0, n).  Copied in by the call; the caller keeps ownership. */
typedef struct {
    int32_t kind;
    int32_t ntarget;
    int32_t target[2];
    int32_t ncontrol;
    int32_t control[2];
    double theta[3];
} qt_gate;

/* Stable gate handle, unique within a circuit and never reused. */
typedef uint64_t qt_gate_id;

/* What one qt_update_state did.  "Partition-passes" count (partition x
 * fused pass) units: the incremental work unit of Section III-E. */
typedef struct {
    int32_t segments_total;      /* checkpoint segments in the plan */
    int32_t segments_run;        /* segments that launched work */
    int32_t passes_total;        /* fused passes in the whole plan */
    int32_t passes_run;          /* fused passes launched */
    int32_t launches;            /* kernel launches issued */
    int32_t gates_total;         /* gates in the circuit */
    int64_t partition_passes_total;     /* sum over all passes of all partitions */
    int64_t partition_passes_run;       /* sum over launched passes of partitions processed */
    double clean_fraction;       /* 1 - run / total partition-passes */
    uint64_t amp_updates;        /* sum over gates of the amplitudes recomputed in the gate's segment
                                    (a full run: gates x 2^n) */
    uint64_t hbm_bytes;          /* algorithmic bytes: 2 x bytes/amp x amplitudes, per pass */
    double host_ms;              /* wall time of the call */
    double gpu_ms;               /* device time of the call's stream work (CUDA events), -1 if not timed */
    double pass_kernel_ms;       /* summed device time of the fused-pass kernels (option kernel_timing) or -1 */
    int32_t pass_kernel_launches;
    int32_t tensor_blocks;       /* tensor-core block ops in the launched passes (complex64, option tc_blocks) */
    uint64_t pass_kernel_bytes;  /* algorithmic bytes of those launches */
    uint64_t h2d_bytes;          /* host-to-device bytes uploaded (fused ops and worklists) */
    uint64_t pass_kernel_alu_ops; /* algorithmic floating-point ops of the timed fused-pass launches
                                     (binary32 ops for QT_C64 and QT_C128_DF, binary64 for QT_C128) */
} qt_update_stats;

/* Create an empty circuit (no levels) whose state is |0...0>.
 * n_qubits in [1, 34]; log2_partition in [max(0, n_qubits - 30), n_qubits]
 * (partition size 2^log2_partition amplitudes, the paper's block size B,
 * Section III-C; at most 2^30 partitions).
 * Allocates host memory only.  *out receives the handle. */
qt_status qt_create(int32_t n_qubits, int32_t dtype, int32_t log2_partition, qt_circuit** out);

/* Free the circuit and all its host and device memory.  NULL is allowed.
 * Waits for the circuit's device work (and an asynchronous read in flight)
 * first.  (No counterpart in the paper: its circuit is a C++ object,
 * Listing 1, freed by its destructor.) */
qt_status qt_destroy(qt_circuit* c);

/* Number of levels (the paper's nets, Section III-B), and of gates over all
 * levels, of the circuit as edited so far (pending edits included).
 * QT_ERR_ARG if c or out is NULL. */
qt_status qt_num_levels(const qt_circuit* c, int32_t* out);
qt_status qt_num_gates(const qt_circuit* c, int64_t* out);

/* Insert an empty level at position pos in [0, num_levels]; levels at and
 * after pos move up by one (insert_net, Table 2). */
qt_status qt_insert_level(qt_circuit* c, int32_t pos);

/* Remove level pos and all its gates (remove_net, Table 2). */
qt_status qt_remove_level(qt_circuit* c, int32_t pos);

/* Add a gate to level `level` (insert_gate, Table 2).  QT_ERR_CONFLICT if it
 * shares a qubit with a gate already in the level; the circuit is then
 * unchanged (Section III-B).  *out receives the new gate's id. */
qt_status qt_insert_gate(qt_circuit* c, int32_t level, const qt_gate* g, qt_gate_id* out);

/* Remove gate `id` from level `level` (remove_gate, Table 2). */
qt_status qt_remove_gate(qt_circuit* c, int32_t level, qt_gate_id id);

/* Replace gate `id` of level `level` by *g (a remove followed by an insert
 * into the same level, checked for conflicts against the other gates).
 * *out receives the new id.  On error nothing changes. */
qt_status qt_replace_gate(qt_circuit* c, int32_t level, qt_gate_id id, const qt_gate* g, qt_gate_id* out);

/* Bring the state up to date with all pending edits (update_state, Table 2).
 * force_full = 0: incremental -- only segments at or after the first edited
 * one run, each over the partitions its edits (or the dirty partitions
 * flowing in from earlier segments) can reach (Section III-E).
 * force_full = 1: every segment over every partition.  Both give the same
 * bits.  Blocks until the device work is done.  stats may be NULL.
 * On error the edits stay pending (so reads return QT_ERR_STALE), and:
 *   - an error raised before any device work is enqueued (QT_ERR_OOM from
 *     mem_limit or a failed allocation, QT_ERR_ARG) leaves the device state
 *     and every checkpoint of the last successful update untouched: undoing
 *     the edits and updating again gives that state back bit for bit
 *     without recomputing it, and otherwise the next update still runs
 *     incrementally from those checkpoints;
 *   - an error during the device work (QT_ERR_CUDA, QT_ERR_TIMEOUT) leaves
 *     the checkpoints the update was rewriting in place unknown: the next
 *     successful update re-simulates the whole circuit. */
qt_status qt_update_state(qt_circuit* c, int32_t force_full, qt_update_stats* stats);

/* Copy amplitudes [first, first + count) of the current state -- the
 * alpha_b of Section II-A, b the index with qubit q at bit q -- to host
 * memory (binary64 re/im pairs for QT_C128 and QT_C128_DF, binary32 pairs
 * for QT_C64).  host_dst holds count x 16 bytes (8 for QT_C64) and stays the
 * caller's.  Blocks until the copy is done.  QT_ERR_STALE while edits are
 * pending or after a failed device update; QT_ERR_RANGE if the range exceeds
 * 2^n; QT_ERR_ARG if host_dst is NULL with count > 0. */
qt_status qt_read_amplitudes(const qt_circuit* c, uint64_t first, uint64_t count, void* host_dst);

/* Same, into a device buffer of the caller (same element format). */
qt_status qt_read_amplitudes_device(const qt_circuit* c, uint64_t first, uint64_t count, void* device_dst);

/* Start the same copy to host memory without waiting for it: the amplitudes
 * are converted into a device snapshot buffer on the circuit's stream (the
 * library allocates it: count x 16 bytes, 8 for QT_C64, kept until
 * qt_release_device or qt_destroy), then copied to host_dst on a second
 * stream, so that edits and the next qt_update_state run while the copy is in
 * flight.  host_dst (best pinned) must stay valid and untouched until
 * qt_read_wait returns; a second call first lets the previous copy finish
 * with the snapshot buffer.  Errors as qt_read_amplitudes, plus QT_ERR_OOM
 * if the snapshot buffer cannot be allocated. */
qt_status qt_read_amplitudes_async(qt_circuit* c, uint64_t first, uint64_t count, void* host_dst);

/* Block until the copy started by the last qt_read_amplitudes_async has
 * arrived in host memory (QT_OK at once if none is in flight). */
qt_status qt_read_wait(qt_circuit* c);

/* sum_b |alpha_b|^2 of the current state (Section II-A), reduced with
 * FP64-class accuracy for every dtype (float-float partial sums, FP64 tree). */
qt_status qt_norm(const qt_circuit* c, double* out);

/* Fidelity |<a|b>|^2 / (<a|a> <b|b>) of the current states of two circuits
 * with the same qubit count (any dtypes; a complex64 result against a
 * complex128 one measures the complex64 drift).  Both must be readable (no
 * pending edits).  FP64-class reduction (float-float partial sums, binary64
 * tree).  Runs on a's stream after waiting for b's. */
qt_status qt_fidelity(const qt_circuit* a, const qt_circuit* b, double* out);

/* Largest amplitude difference max_b |alpha_b - beta_b| between the current
 * states of two circuits with the same qubit count (any dtypes), computed
 * in binary64 on the device (each amplitude converted to binary64: binary32
 * exactly, float-float as hi + lo).  Against a complex128 run of the same
 * gates it measures the complex64 rounding error per amplitude, the
 * quantity the max-abs tolerance bounds.  Both states must be readable.
 * Runs on a's stream after waiting for b's.  (No counterpart in the paper,
 * which states no precision.) */
qt_status qt_max_abs_diff(const qt_circuit* a, const qt_circuit* b, double* out);

/* Marginal probabilities of the k <= 10 qubits qubits[0..k-1] in the current
 * state: out[v] (2^k doubles, host memory) = sum of |alpha_b|^2 over the
 * indices b whose bit qubits[j] equals bit j of v (squared amplitudes are
 * the probabilities of the basis states, Section II-A).  FP64-class. */
qt_status qt_probabilities(const qt_circuit* c, int32_t k, const int32_t* qubits, double* out);

/* qt_norm_static -- the norm of amplitudes the caller holds in device memory,
 * computed without allocating anything.  (The paper has no counterpart: this
 * entry point serves callers that cannot let a library call cudaMalloc, such
 * as a process that routes all device memory through its own allocator or
 * pool, or a latency-critical loop that cannot afford an allocation and the
 * synchronisation it may imply.)
 *
 * amps_device: `count` amplitudes in device memory, in the element format of
 *   `dtype` (QT_C128: binary64 re, im; QT_C64: binary32 re, im; QT_C128_DF:
 *   binary32 re_hi, re_lo, im_hi, im_lo).  Not modified.
 * out_device: one double in device memory; receives sum |a|^2, reduced like
 *   qt_norm (float-float partial sums, binary64 tree).  Written by the work
 *   enqueued on `cuda_stream` (a cudaStream_t, NULL = the legacy default
 *   stream); the call does not wait for it.
 * count: 1 <= count <= QT_NORM_STATIC_MAX_AMPS, else QT_ERR_RANGE.
 * Memory: the partial sums live in one file-scope device array of
 *   QT_NORM_STATIC_SCRATCH_BYTES bytes (1216 doubles), which every GPU that
 *   loads the library holds until the process exits.  Every call looks up
 *   that array's address on the current device (cudaGetSymbolAddress, which
 *   allocates nothing), so a context reset between calls does no harm; the
 *   first call on a device may load the library's device code, so make it
 *   before any stream capture.  The call never calls cudaMalloc, cudaFree or
 *   any allocating routine.
 * Sharing: all calls share the one array, and it keeps the last call's
 *   contents (each call overwrites every partial sum it reads, so nothing
 *   needs clearing); two calls whose work overlaps on the GPU (on different
 *   streams, say) race on it and must be ordered by the caller.
 * Errors: QT_ERR_ARG (NULL pointer, unknown dtype), QT_ERR_RANGE (count),
 *   QT_ERR_CUDA (address lookup or launch failed); the message is in
 *   qt_last_error(NULL). */
#define QT_NORM_STATIC_MAX_AMPS ((uint64_t)1 << 34)
#define QT_NORM_STATIC_SCRATCH_BYTES 9728
qt_status qt_norm_static(const void* amps_device, uint64_t count, int32_t dtype, double* out_device,
                         void* cuda_stream);

/* Tuning options.  The paper's one knob is the block size B (Section IV,
 * "Impact of Block Size"), here log2_partition of qt_create; the checkpoint
 * options choose how many of Section III-F's per-net state vectors are kept;
 * the others have no counterpart in the paper.  QT_ERR_ARG for an unknown key
 * or a value out of range; the circuit is then unchanged.
 * Options (value semantics):
 *   "ckpt_interval"  levels per checkpoint segment (>= 1; default 4)
 *   "ckpt_budget"    > 0: bytes of device memory for the state and its
 *                    checkpoints (one state vector each); the interval is
 *                    then the smallest whose checkpoints fit (Section III-F's
 *                    per-net states, as many as the memory holds), kept across
 *                    updates while it still fits; 0 (default): ckpt_interval
 *   "fusion"         0: one gate per pass; 1: tile fusion (default)
 *   "tile_high"      max qubits at or above the tile's low bits per pass (0..7)
 *   "mem_limit"      device-memory budget in bytes for state + checkpoints (0 = none)
 *   "kernel_timing"  1: time every fused-pass kernel with CUDA events (stats)
 *   "tma"            1: persistent register kernel that stages the next tile with
 *                    bulk copies (cp.async.bulk + mbarrier, bounded waits: a wait
 *                    that expires makes qt_update_state return QT_ERR_TIMEOUT);
 *                    0 (default): one CTA per tile
 *   "test_stall_staging"  1 (with "tma" = 1): the staging copies are withheld, so
 *                    the kernel's bounded wait expires after 1 s and the update
 *                    returns QT_ERR_TIMEOUT; a failure-detection test hook
 *   "reg_kernel"     1: register-resident pass kernel for tiles of 2^7 amplitudes or more
 *                    (default); 0: shared-memory pass kernel for every tile
 *   "tc_blocks"      complex64 only: 1 = fold runs of a pass's ops that act on at most
 *                    five tile qubits into one 32x32 block applied on the tensor cores
 *                    (tcgen05 MMA, 3xTF32: fp32-class accuracy) inside the fused pass
 *                    (tiles of 12 qubits); 0 (default) = every op in the register kernel
 *   "tc_threshold"   tenths of a dense one-qubit op: a run becomes a block when the
 *                    register kernel's estimated cost of its ops exceeds this
 *                    (default 40); 0 makes every run a block
 *   "dry_run"        1: qt_update_state plans and tracks but launches nothing and
 *                    allocates nothing (host-logic testing); the device state is
 *                    marked stale and the next real update runs in full.
 * Changing ckpt_interval, fusion, tile_high, tc_blocks or tc_threshold (or a
 * budget that changes the interval) makes the next update full. */
qt_status qt_set_option(qt_circuit* c, const char* key, int64_t value);

/* Run the circuit's GPU work on `cuda_stream` (a cudaStream_t; NULL = the
 * library's own stream).  The caller keeps ownership of the stream and must
 * keep it alive while the circuit uses it.  (No counterpart in the paper,
 * whose runtime is CPU-only.) */
qt_status qt_set_stream(qt_circuit* c, void* cuda_stream);

/* Introspection of the last qt_update_state (real or dry run), for tests and
 * debugging.  For segment `seg`: levels [*first_level, *first_level +
 * *nlevels); optional out arrays of 2^(n - log2_partition) bytes receive the
 * segment's forward dirty set F (partitions whose output may have changed)
 * and worklist W (partitions recomputed), 1 = member. */
qt_status qt_num_segments(const qt_circuit* c, int32_t* out);
qt_status qt_segment_info(const qt_circuit* c, int32_t seg, int32_t* first_level, int32_t* nlevels,
                          int32_t* npasses, uint8_t* dirty_out, uint8_t* worklist_out);

/* Partitions that segment `seg` of the current plan can change: the union of
 * its passes' supports (the partitions where every control and phase
 * condition above the partition bits can hold; Section III-D).  On every
 * other partition the state after the segment equals the state before it,
 * so a copy-on-write checkpoint store (Section III-F) could share those
 * partitions with the previous checkpoint.  touched_out: 2^(n -
 * log2_partition) bytes, 1 = member.  Valid after a qt_update_state (real or
 * dry run); QT_ERR_RANGE for a segment out of range. */
qt_status qt_segment_touched(const qt_circuit* c, int32_t seg, uint8_t* touched_out);

/* Message of the last failed call on c (or of the last failed qt_create,
 * qt_norm_static or batch call on this thread when c is NULL).  Valid until
 * the next call on c.  (No counterpart in the paper: its modifiers throw a
 * C++ exception on a conflicting gate, Section III-B; no exception crosses
 * this ABI.) */
const char* qt_last_error(const qt_circuit* c);

/* Free the circuit's device memory (state, checkpoints, buffers) and keep
 * its circuit; the next qt_update_state re-simulates in full. */
qt_status qt_release_device(qt_circuit* c);

/* Device bytes the circuit currently holds for its state and checkpoints. */
qt_status qt_device_bytes(const qt_circuit* c, int64_t* out);

/* ------------------------------------------------------------ batches ---
 * Many small circuits (10 or more qubits each; tiles of 2^10-2^12
 * amplitudes) simulated together in ONE persistent launch: the tiles of all
 * circuits' passes are dequeued in wavefront order and each waits (bounded,
 * 1 s; QT_ERR_TIMEOUT if it expires) only for the previous pass of its own
 * circuit.  A run re-simulates every circuit in full from |0...0> with its
 * current gates (edits are made on the circuits with the usual calls) into
 * the batch's own device arena; the circuits' own states are untouched.
 * From the second run with an unchanged structure the whole run is a CUDA
 * graph replay; parameter edits (new angles) keep the structure. */
typedef struct qt_batch qt_batch;

typedef struct {
    double gpu_ms;            /* device time of the run (CUDA events) */
    int32_t circuits;
    int32_t passes;           /* fused passes over all circuits */
    int32_t tiles;            /* work items of the persistent launch */
    int32_t graph_replayed;   /* 1: the run replayed the captured graph */
    uint64_t amp_updates;     /* sum over circuits of gates x 2^n */
} qt_batch_stats;

/* All circuits must share one dtype.  The batch references the circuits
 * (the caller keeps them alive and unchanged during qt_batch_run). */
qt_status qt_batch_create(qt_circuit* const* circuits, int32_t count, qt_batch** out);
qt_status qt_batch_run(qt_batch* b, qt_batch_stats* stats);
/* Amplitudes of circuit `index` from the last run (format as qt_read_amplitudes). */
qt_status qt_batch_read_amplitudes(const qt_batch* b, int32_t index, uint64_t first, uint64_t count,
                                   void* host_dst);
qt_status qt_batch_destroy(qt_batch* b);
/* Message of the batch's last failed call. */
const char* qt_batch_last_error(const qt_batch* b);

/* ------------------------------------------------------------ serving ---
 * A request is a short list of circuit edits followed by an incremental
 * update of one circuit -- the paper's incremental iteration, Section IV-C.
 * The server runs requests on `workers` host threads; every circuit has its
 * own CUDA stream, so requests on different circuits overlap on the GPU, and
 * a request arriving while others run starts as soon as a worker and device
 * memory are free (continuous batching).  Device memory (state plus
 * checkpoints of every resident circuit) is admitted against
 * hbm_budget_bytes (0 = no budget): a request whose circuit is not resident
 * and does not fit evicts idle circuits least-recently-used first
 * (qt_release_device), or waits while other requests proceed.  Requests on
 * one circuit run in submission order.  With a budget, the server also sets
 * every circuit's "ckpt_budget" option to its share of the budget (the
 * budget less one spare state vector per circuit, divided in proportion to
 * state size, at least two state vectors each), so that circuits stay
 * resident rather than being evicted and re-simulated; each qt_server_add_
 * circuit re-divides it.  The caller keeps ownership of the circuits and
 * must not call into a circuit while the server may use it. */
typedef struct qt_server qt_server;

typedef enum {
    QT_EDIT_INSERT_LEVEL = 0, /* level */
    QT_EDIT_INSERT_GATE = 1,  /* level, gate */
    QT_EDIT_REMOVE_GATE = 2,  /* level, id */
    QT_EDIT_REPLACE_GATE = 3, /* level, id, gate */
    QT_EDIT_REMOVE_LEVEL = 4  /* level */
} qt_edit_kind;

typedef struct {
    int32_t kind;
    int32_t level;
    qt_gate_id id;
    qt_gate gate;
} qt_edit;

typedef struct {
    int32_t status;          /* qt_status of the request */
    int32_t circuit;         /* slot */
    double queue_ms;         /* submit -> start (waiting for a worker, the circuit or memory) */
    double service_ms;       /* start -> done */
    double latency_ms;       /* submit -> done */
    qt_update_stats stats;   /* of the request's qt_update_state */
    int32_t n_new_ids;       /* ids created by the request's inserts and replaces, in order */
    int32_t reserved;
    qt_gate_id new_ids[8];
} qt_request_result;

qt_status qt_server_create(int32_t workers, int64_t hbm_budget_bytes, qt_server** out);
/* Runs every queued request, then stops the workers and frees the server. */
qt_status qt_server_destroy(qt_server* s);
qt_status qt_server_add_circuit(qt_server* s, qt_circuit* c, int32_t* slot);
/* Queue a request (edits are copied); *ticket identifies it. */
qt_status qt_server_submit(qt_server* s, int32_t slot, int32_t nedits, const qt_edit* edits, uint64_t* ticket);
/* Block until the request is done, copy its result and forget the ticket. */
qt_status qt_server_wait(qt_server* s, uint64_t ticket, qt_request_result* out);
/* Device bytes admitted for resident circuits, evictions so far, requests queued. */
qt_status qt_server_info(qt_server* s, int64_t* resident_bytes, int32_t* evictions, int32_t* queued);

#ifdef __cplusplus
}
#endif

#endif /* QTASK_H */
