// qt_internal.h -- internal types shared by the host engine and the kernels
// of libqtask.so.  Not part of the public ABI (include/qtask.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "qtask.h"

namespace qt {

constexpr int kMaxQubits = 34;
constexpr int kMaxTileHigh = 7;      // tile qubits above the contiguous low run
constexpr int kMaxRegBits = 5;       // register-index bits of the register kernel (32 amplitudes a thread)
constexpr int kThreads = 256;        // threads per fused-pass CTA

// ------------------------------------------------------------------ ops --
// A gate lowers to one primitive op; a fused pass is a sequence of ops applied
// to one tile of amplitudes held in shared memory (see qt_kernels.cu).
enum OpKind : int32_t {
    OP_DENSE = 0,  // general complex 2x2 on target q0
    OP_REAL = 1,   // real 2x2 on target q0
    OP_DIAG = 2,   // diag(d0, d1) on q0 (q0 may lie outside the tile: uniform factor)
    OP_PHASE = 3,  // multiply by f where every bit of cmask is 1 (Z S T CZ CP, fused phases)
    OP_X = 4,      // exchange the pair on target q0
    OP_ANTI = 5,   // [[0, m01], [m10, 0]] on target q0 (Y and fused permutation-phases)
    OP_SWAP = 6,   // exchange amplitudes with (q0, q1) bits (1,0) and (0,1)
    // (7 is OP_PERM, a register-kernel layout change)
    OP_IREAL = 8,  // [[a, ib], [ic, d]] with a, b, c, d real on target q0 (RX and its products)
    OP_BLOCK = 9,  // a 32x32 unitary on five tile qubits (Pass::blocks[q0]), applied on the tensor cores
};

// Phase sub-kinds, chosen on the host so that exact factors cost no rounding.
enum PhaseKind : int32_t { PH_GENERAL = 0, PH_NEG = 1, PH_POS_I = 2, PH_NEG_I = 3 };

struct HostOp {
    int32_t kind = OP_DENSE;
    int32_t q0 = -1, q1 = -1;  // target qubits
    uint64_t cmask = 0;        // qubits that must all be 1 (controls; for PHASE also the phase qubits)
    double m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // DENSE/REAL: (m00, m01, m10, m11) as re,im pairs.  DIAG: d0 = m[0..1], d1 = m[2..3].
    // PHASE: f = m[0..1].  ANTI: m01 = m[0..1], m10 = m[2..3].
    int32_t ngates = 1;        // original gates folded into this op
};

// Public gate record as stored by the circuit.
struct Gate {
    qt_gate g;
    qt_gate_id id;
};

struct Level {
    std::vector<Gate> gates;  // kept in canonical order (ascending lowest qubit)
};

// ---------------------------------------------------------------- plans --
// A fused block: the product of a run of ops acting only on five tile qubits
// q[0..4] (block-index bit i = qubit q[i]), as a 32x32 complex matrix u
// (row-major, re/im interleaved: 2048 doubles), built in FP64 on the host.
struct Block {
    int32_t q[5];
    std::vector<double> u;
};

struct Pass {
    std::vector<HostOp> ops;
    int32_t lt = 0;                 // tile low bits: amplitudes [0, 2^lt) are contiguous
    int32_t nh = 0;                 // tile qubits at or above lt
    int32_t h[kMaxTileHigh] = {0};  // those qubits, ascending
    uint32_t M = 0;                 // partition-index bits spanned by the tile (coupling)
    std::vector<uint32_t> supp_masks;  // partition q is touched iff (q & m) == m for some m
    bool supp_all = false;
    int32_t ngates = 0;
    std::vector<Block> blocks;      // OP_BLOCK ops (complex64 tensor-core path)
    bool same_as(const Pass& o) const;
};

struct SegPlan {
    int32_t first_level = 0, nlevels = 0;
    std::vector<Pass> passes;
};

struct PlanParams {
    int n = 0, p = 0;
    int lt = 0;        // tile low bits
    int nh_max = 0;    // tile qubits allowed at or above lt
    bool fusion = true;
    bool merge = true;  // multiply consecutive one-qubit ops on a qubit into one 2x2
    // complex64 only: fold runs of ops on at most five tile qubits into
    // tensor-core blocks when their estimated register-kernel cost exceeds
    // tc_threshold (in units of one dense one-qubit op)
    bool tc_blocks = false;
    double tc_threshold = 4.0;
};

// Fold runs of a pass's ops into tensor-core blocks (complex64; tiles of 12
// qubits: lt = 7 low and 5 high).  Ops that commute with the block being
// built (no common qubit) may be moved ahead of it.
void fuse_blocks(Pass* ps, const PlanParams& pp);
// Operand B of a block (64 x 64 real embedding of u, tf32 hi and lo in the
// MMA's 128-byte-swizzled K-major shared-memory layout): kBlockBytes bytes.
void block_operand(const Block& b, float* out);

// Lower one public gate to primitive ops (A2: gate matrices and classification).
bool lower_gate(const qt_gate& g, int n, std::vector<HostOp>* out, std::string* err);
// Validate a gate against the circuit's qubit count.
bool check_gate(const qt_gate& g, int n, std::string* err);
uint64_t gate_qubit_mask(const qt_gate& g);

// Plan one segment: canonical gate list -> fused passes (A3).
SegPlan plan_segment(const std::vector<const qt_gate*>& gates, const PlanParams& pp);

// Partition bitsets (A6).
struct Bitset {
    std::vector<uint64_t> w;
    uint32_t nbits = 0;
    void resize(uint32_t n) { nbits = n; w.assign((n + 63) / 64, 0); }
    bool get(uint32_t i) const { return (w[i >> 6] >> (i & 63)) & 1; }
    void set(uint32_t i) { w[i >> 6] |= uint64_t(1) << (i & 63); }
    void fill() {
        for (auto& x : w) x = ~uint64_t(0);
        trim();
    }
    void trim() {
        if (nbits & 63) w.back() &= (uint64_t(1) << (nbits & 63)) - 1;
    }
    bool any() const {
        for (auto x : w)
            if (x) return true;
        return false;
    }
    bool all() const;
    uint64_t count() const;
    bool or_with(const Bitset& o);  // returns true if anything changed
};

Bitset pass_support(const Pass& ps, uint32_t nparts);
// D := D u { q ^ m : q in D n supp, m in span(M) }
void close_forward(Bitset* D, const Pass& ps, const Bitset& supp);
// Smallest W containing F that is closed under every pass's coupling.
void close_all(Bitset* W, const std::vector<Pass>& passes, const std::vector<Bitset>& supps);

// ------------------------------------------------------- device encoding --
// One op as the kernels read it (128 bytes).  Matrix entries are stored in
// the arithmetic of the circuit's dtype: binary64 (QT_C128), binary32
// (QT_C64) or float-float (hi, lo) pairs (QT_C128_DF).
//
// Two kernels read it.  The shared-memory kernel (small tiles) walks the
// op's index pattern (fixpos/fixval).  The register kernel (tiles of 2^7 and
// more) keeps each thread's amplitudes in registers: tile bits 0-4 are the
// lane bits, the other tile bits are split between register-index bits and
// warp bits by the current layout; OP_PERM ops change the layout through
// shared memory so that every target is a lane or register bit when its op
// runs.  The layout planner resolves every op against the layout it runs in
// and writes the result to DevOp::rh.
enum : int32_t { OP_PERM = 7 };  // register-kernel layout change

// Where a tile's bits sit in the register kernel: the tile bit held by each
// lane-id bit, register-index bit and warp-id bit, and the pending flip.  A
// thread's amplitude at physical slot P (its lane, register index and warp)
// is the tile's amplitude at index L(P) ^ flip: uncontrolled X gates only
// toggle flip and uncontrolled SWAP gates only exchange two entries, so
// neither moves data; the next layout change or the final store applies
// both.
struct TileLayout {
    int8_t lane[5];
    int8_t reg[5];
    int8_t warp[3];
    int8_t pad[3];
    uint32_t flip;
};
static_assert(sizeof(TileLayout) == 20, "TileLayout layout");

// Register-kernel dispatch code of an op: its kind and where its qubits sit
// in the thread's layout (register bit 0 after the rename, a lane bit, a bit
// held by the thread or outside the tile), chosen on the host so that the
// kernel takes one branch per op.
enum RegCode : uint8_t {
    RC_PERM = 0,
    RC_DENSE_R, RC_DENSE_L,  // _R: target on register bit 0 (DENSE: bit b), _L: on lane bit a
    RC_REAL_R, RC_REAL_L,
    RC_ANTI_R, RC_ANTI_L,
    RC_IREAL_R, RC_IREAL_L,
    RC_X_R, RC_X_L,
    RC_SWAP_RR,  // register bits a < b
    RC_SWAP_LR,  // lane bit a, register bit b
    RC_SWAP_LL,  // lane bits a, b
    RC_DIAG_G,   // qubit a outside the tile: one factor per tile
    RC_DIAG_T,   // thread-index bit a (lane bits 0-4, warp bits 5-7): one factor per thread
    RC_DIAG_R,   // register bit a
    RC_PH_NEG, RC_PH_POS_I, RC_PH_NEG_I, RC_PH_GEN,
    RC_PH_GROUP,  // consecutive phases merged: DevOp::b1 terms (PhTerm) in the slots that follow
    RC_NOP,
    RC_MMA        // fused block on the tensor cores (BlockStage in DevOp::m)
};

// Everything the register kernel reads per op besides cm_glob and the
// matrix, in one 16-byte load.  Conditions are on physical bits: the thread
// index (lane bits 0-4, warp bits 5-7) and the register index; an op applies
// where (bits ^ value) & mask == mask, the value marking conditions on
// flipped tile bits.
struct RegHdr {
    uint8_t code;     // RegCode
    int8_t ren;       // > 0: exchange register bits 0 and ren before the op (pair ops)
    int8_t a, b;      // code-specific bits (see RegCode)
    uint16_t cm_reg;  // conditions among register-index bits
    uint8_t mcls;     // PHASE: 0 no register condition, 1 exactly one unflipped (bit in a), 2 otherwise
    uint8_t cv_reg;   // flipped register conditions
    uint32_t cm_thr;  // conditions among thread-index bits
    uint32_t cv_thr;  // flipped thread conditions
};
static_assert(sizeof(RegHdr) == 16, "RegHdr layout");

struct DevOp {
    int32_t kind;
    int32_t b0;        // tile-local bit of target q0 (-1: q0 outside the tile; DIAG only)
    int32_t b1;        // tile-local bit of q1 (SWAP)
    int32_t gq;        // global qubit q0 (DIAG outside the tile)
    uint64_t cm_glob;  // control bits outside the tile (global index positions)
    int8_t fixpos[6];  // tile-local bits fixed by the op's index pattern, ascending
    uint8_t nfix;      // number of fixed bits; the op visits 2^(tile bits - nfix) indices
    uint8_t fixval;    // bit k = value of fixpos[k]
    uint32_t cm_tile;  // control bits inside the tile (tile-local positions)
    int8_t sub;        // PhaseKind (PHASE)
    int8_t nreg, nwarp;  // OP_PERM: register bits and warp bits of the new layout
    int8_t pad0;
    int8_t perm[8];    // OP_PERM: tile bit of register bit k (k < nreg), then of warp bit w, in the
                       // new layout (lane bit i holds tile bit i); m holds the old TileLayout
    RegHdr rh;         // register kernel (filled by the layout planner)
    union {
        double d[8];
        float f[16];
    } m;
};
static_assert(sizeof(DevOp) == 128 && offsetof(DevOp, rh) == 48 && offsetof(DevOp, m) == 64, "DevOp layout");

// One phase of a merged group (RC_PH_GROUP), four to a DevOp slot after the
// group's header.  A thread multiplies together the factors of a step's
// terms whose conditions hold for it (outside the tile: the tile base's bits
// in cm_glob are 1; thread index: (tid ^ cv_thr) & cm_thr == cm_thr), then
// multiplies the product into its amplitudes of the step's class: all of
// them (mcls 0) or those whose register index has bit k set (mcls 1).
struct PhTerm {
    union {
        double d[2];
        float f[4];
    } f;               // the factor, encoded like entry 0 of DevOp::m
    uint64_t cm_glob;
    uint16_t cm_thr, cv_thr;
    uint8_t last;      // last term of its step
    uint8_t mcls, k;   // the step's registers
    uint8_t pad;
};
static_assert(sizeof(PhTerm) == 32, "PhTerm layout");
constexpr int kTermsPerSlot = int(sizeof(DevOp) / sizeof(PhTerm));
// Ops the register kernel stages in shared memory at a time; a merged
// group's header and its term slots never straddle two chunks.
constexpr int kOpChunk = 64;

// The tensor-core block op (RC_MMA) as the register kernel reads it, in
// DevOp::m.  The 4096-amplitude tile is the MMA operand A: row m (128) = the
// seven tile bits outside the block, column 2b + {re, im} (64) = block index
// b.  A thread's amplitude at physical slot (lane, register, warp) has row
// and block index given by XOR-ing the contributions of its set physical
// bits and of the pending flip (all linear over GF(2)); so has its byte
// offset in the swizzled operand (block_a_offset), whose bit fields (block
// bit 4; row bits 3-6; row bits 0-2; block bits 1-3 XOR row bits 0-2; block
// bit 0) sit at disjoint positions.  The op holds those offset
// contributions.  After the op the layout is fixed: lane bit i = row bit i,
// warp bits 0-1 = row bits 5-6, register bit k = block bit k, warp bit 2 =
// block bit 4.
struct BlockStage {
    int64_t boff;     // byte offset of the block's operand B (tf32 hi, then lo; 32 KB)
    int8_t s[5];      // tile bit of block bit i
    int8_t rows[7];   // tile bit of row bit i
    uint16_t a_lane[5], a_reg[4], a_warp[3], a_flip;  // operand-A byte-offset contributions
};
static_assert(sizeof(BlockStage) <= 64, "BlockStage fits DevOp::m");
// Byte offset of element (row m, column 2 kb) of the operand-A layout:
// K-major fp32, two 32-column K atoms of 128 rows x 128 B, 16-byte chunks
// swizzled by the row's low three bits (XOR-linear in the bits of m and kb).
constexpr uint32_t block_a_offset(uint32_t m, uint32_t kb) {
    return ((2u * kb) >> 5) * 16384u + (m >> 3) * 1024u + (m & 7u) * 128u +
           (((((2u * kb) & 31u) >> 2) ^ (m & 7u)) << 4) + (((2u * kb) & 3u) << 2);
}
constexpr int kBlockBytes = 32768;  // operand B of one block: 64 x 64 tf32, hi and lo

struct DevPass {
    int32_t p;             // log2 partition size
    int32_t lt;            // tile low bits
    int32_t nh;            // tile high qubits
    int32_t nins;          // tile high qubits below p (zeros inserted into the tile counter)
    int32_t h[kMaxTileHigh];
    int32_t ins[kMaxTileHigh];
    int32_t tpg_log2;      // log2 tiles per partition group
    int32_t nops;
    uint32_t M;            // partition-index coupling mask
    int32_t npart_log2;    // log2 number of partitions
    int64_t op_offset;     // into the device op array
    int32_t reg_kernel;    // 1: register kernel with the initial layout below
    int32_t nreg, nwarp;   // register-index bits and warp bits (lane bits = 5)
    int32_t layout[8];     // tile bit of register bit k (k < nreg), then of warp bit w
    int32_t tma;           // 1: persistent register kernel with bulk-copy (TMA) staging
    int32_t test_stall;    // 1: withhold the staging copies so the bounded wait expires (test hook)
    int32_t groups;        // 1: the ops hold merged phase groups (RC_PH_GROUP)
    TileLayout fin;        // register kernel: the layout the tile is stored from
    int32_t mma;           // 1: the ops hold tensor-core blocks (RC_MMA)
    int32_t pad_mma;
    const unsigned char* blk;  // device buffer of the blocks' B operands (mma passes)
    // register kernel: amplitude-index offset of each register bit's tile bit
    // in the initial layout (rin) and the final layout (rout); an amplitude's
    // index is the thread's index XOR the offsets of its register-index bits
    uint64_t rin[kMaxRegBits];
    uint64_t rout[kMaxRegBits];
};

// Register-kernel layout planning for one pass (host): fills the initial
// layout of dp and rewrites the ops' roles, inserting OP_PERM where needed.
// coef_bytes: size of one complex matrix entry (16 for binary64 and
// float-float, 8 for binary32), for exchanging entries when an op's target
// is flipped.
// reorder: let commuting ops whose targets are placed run before ops that
// need a layout change.
// phase_groups: merge runs of phases into RC_PH_GROUP ops where that is
// estimated to save work (sets dp->groups).
// dense_regk: a DENSE op whose target sits on register bit k > 0 keeps it
// there (RegHdr::b = k; the kernel pairs registers across bit k) instead of
// exchanging register bits 0 and k first (complex64, where the exchange's
// moves are a large share of the op).
void plan_register_layout(DevPass* dp, std::vector<DevOp>* ops, int coef_bytes, bool reorder = true,
                          bool phase_groups = true, bool dense_regk = false);

// Fill dp->rin / dp->rout from the planned layouts (needs lt and h).
void set_register_offsets(DevPass* dp);

// Kernel launchers (qt_kernels.cu).  Return a cudaError_t as int.
// err: device int set to 1 when a bounded wait of the TMA-staged kernel
// expires (may be null: that kernel is then not used).
int launch_pass(int dtype, void* dst, const void* src, const DevPass& dp, const DevOp* ops,
                const uint32_t* worklist, uint32_t ngroups, int* err, void* stream);
int launch_pass_reg(int dtype, void* dst, const void* src, const DevPass& dp, const DevOp* ops,
                    const uint32_t* worklist, uint32_t ngroups, int* err, void* stream);
// The same for passes with merged phase groups (dp.groups; qt_pass_grp.cu).
int launch_pass_reg_groups(int dtype, void* dst, const void* src, const DevPass& dp, const DevOp* ops,
                           const uint32_t* worklist, uint32_t ngroups, int* err, void* stream);
int launch_copy_parts(int dtype, void* dst, const void* src, int p, const uint32_t* parts, uint32_t nparts,
                      void* stream);
int launch_init_zero_state(int dtype, void* state, uint64_t namps, void* stream);
int launch_read_convert(int dtype, void* dst, const void* state, uint64_t first, uint64_t count, void* stream);
int launch_norm(int dtype, const void* state, uint64_t namps, double* partials, int npartials, double* out_dev,
                void* stream);
int norm_partials_needed(uint64_t namps);
// Most partial sums launch_norm uses (8 per SM of a 152-SM GB300); the
// no-allocation norm sizes its file-scope array to this.
constexpr int kMaxNormPartials = 152 * 8;
// Streaming multiprocessors of the current device (queried once per device).
int device_sm_count();
// Message for qt_last_error(NULL) on this thread.
void set_thread_error(const std::string& msg);

// Serving-loop hooks (qt_api.cpp): device bytes a circuit holds, bytes its
// next update needs, and releasing its device memory (next update is full).
size_t circuit_device_bytes(const qt_circuit* c);
size_t circuit_state_bytes(const qt_circuit* c);
size_t circuit_device_need(const qt_circuit* c);
void circuit_release_device(qt_circuit* c);

// Batched runs (qt_batch.cpp): the whole circuit planned as one segment with
// one partition, and the device encoding of an op.
void circuit_plan_whole(const qt_circuit* c, std::vector<Pass>* passes, int* dtype, int* n);
DevOp encode_device_op(int dtype, const Pass& ps, const HostOp& op);
// The same, for passes with tensor-core blocks: a block's operand B is
// appended to *blkbuf and the op records its byte offset.
DevOp encode_device_op(int dtype, const Pass& ps, const HostOp& op, std::vector<float>* blkbuf);

// One pass of one circuit in a batched launch.  Work items (tiles) of all
// passes are numbered in wavefront order: every tile of a circuit's pass i
// comes after every tile of its pass i-1.
struct BatchPass {
    DevPass dp;
    uint64_t state_off;   // first amplitude of the circuit's state in the batch arena
    uint32_t first_item;  // global index of the pass's first tile
    uint32_t ntiles;
    int32_t dep;          // counter of the circuit's previous pass (-1: none)
    uint32_t dep_need;    // tiles that counter must reach
    int32_t counter;      // this pass's counter
    int32_t pad;
};
// Persistent batched launch: every CTA takes tiles in order, waits (bounded,
// 1 s) until the previous pass of the tile's circuit is complete, runs the
// tile in place and counts it done.  err is set if a wait expires.
int launch_batch(int dtype, void* arena, const BatchPass* passes, int npasses, const DevOp* ops,
                 uint32_t total_items, uint32_t* head, uint32_t* counters, int* err, size_t smem_bytes,
                 void* stream);
int launch_batch_init(int dtype, void* arena, uint64_t arena_amps, const uint64_t* firsts, int count, void* stream);

// Reductions (qt_reduce.cu).
struct QubitList {
    int32_t k;       // number of qubits (<= 10)
    int32_t q[10];   // bit j of a bin is bit q[j] of the amplitude index
};
int reduce_blocks(uint64_t n);
// out4 (device) receives Re<a|b>, Im<a|b>, <a|a>, <b|b>; partials: 4 per block.
int launch_fidelity(int da, const void* a, int db, const void* b, uint64_t n, double* partials, int nblocks,
                    double* out4, void* stream);
// out (device, one double) receives max_i |a_i - b_i|^2 in binary64;
// partials: one per block.
int launch_max_sq_diff(int da, const void* a, int db, const void* b, uint64_t n, double* partials, int nblocks,
                       double* out, void* stream);
// out (device, 2^k doubles): probability of each value of the listed qubits;
// partials: 2^k per block.
int launch_probabilities(int dtype, const void* s, uint64_t n, const QubitList& ql, double* partials, int nblocks,
                         double* out, void* stream);
size_t bytes_per_amp(int dtype);
// Encode a host op for the device (matrix entries in the dtype's arithmetic).
void encode_matrix(int dtype, const HostOp& op, DevOp* out);

}  // namespace qt
