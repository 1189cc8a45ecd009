// qt_api.cpp -- the C ABI of libqtask.so (include/qtask.h): circuit store and
// modifiers, checkpoint store, dirty-partition tracker and scheduler.
//
// qTask references: programming model and modifiers, Section III-B and
// Table 2; a modifier that makes a gate share a qubit with its net throws,
// Section III-B; frontiers (inserted gates' partitions, successors of removed
// ones) and reachable partitions, Section III-E; per-net state vectors kept
// for incrementality, Section III-F.
//
// Design (GB300): the circuit is cut into segments of `ckpt_interval`
// levels; the state at every segment boundary is a device-resident
// checkpoint slab.  Each segment is planned into fused passes (qt_plan.cpp).
// On update, a segment whose plan and input are unchanged is skipped; for the
// others the tracker seeds the partitions touched by the passes that differ
// between the old and new plan, propagates them forward through the coupling
// of every pass (the forward cone F = partitions whose output may change) and
// closes F under all couplings of the segment (the worklist W).  The
// segment's first pass reads checkpoint s and writes checkpoint s+1 for the
// groups of W, later passes run in place on checkpoint s+1.  Partitions
// outside W keep their bits, partitions of W \ F are recomputed to the same
// bits, so the result equals a full re-simulation bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "qt_internal.h"

using namespace qt;

namespace {
thread_local std::string g_create_error;
}  // namespace

void qt::set_thread_error(const std::string& msg) { g_create_error = msg; }

namespace {

int tile_low_default(int dtype) { return dtype == QT_C64 ? 7 : 6; }

struct Launch {
    int kind;  // 0 = pass, 1 = copy partitions
    int seg;
    int64_t pass_idx;
    DevPass dp;
    size_t wl_offset;  // into the worklist buffer (in entries)
    uint32_t ngroups;
    bool null_worklist;
    bool out_of_place;
    uint64_t parts_processed;
    int ngates;
    double alu_per_amp;  // algorithmic arithmetic ops per amplitude of the pass
    int nblocks;         // tensor-core block ops of the pass
};

// Floating-point operations per amplitude that an op's arithmetic needs (the
// formulas of qt_arith.cuh): float-float -- a 4-term dot product is 43 binary32
// ops, a 2-term one 19, two per complex amplitude; binary32 / binary64 -- a
// complex 2x2 row is 8 ops per amplitude, a real row, a complex multiply 4.
// Phases count only the amplitudes whose condition bits are all 1;
// permutations and exact phases (-1, +-i) need no arithmetic.
double op_alu_per_amp(int dtype, const HostOp& op) {
    const bool df = dtype == QT_C128_DF;
    switch (op.kind) {
        case OP_DENSE: return df ? 86.0 : 8.0;
        case OP_REAL: case OP_IREAL: case OP_DIAG: case OP_ANTI: return df ? 38.0 : 4.0;
        case OP_PHASE: {
            const bool exact = (op.m[0] == -1.0 && op.m[1] == 0.0) || (op.m[0] == 0.0 && (op.m[1] == 1.0 || op.m[1] == -1.0));
            if (exact) return 0.0;
            return (df ? 38.0 : 4.0) / double(uint64_t(1) << __builtin_popcountll(op.cmask));
        }
        default: return 0.0;
    }
}
}  // namespace

struct qt_circuit {
    int n = 0, p = 0, dtype = 0;
    std::vector<Level> levels;
    qt_gate_id next_id = 1;
    bool pending = false;

    // options
    int ckpt_interval = 4;
    int64_t ckpt_budget = 0;  // > 0: bytes for the state and checkpoints; sets the interval
    bool fusion = true;
    bool merge = true;
    int tile_high = 5;  // tiles of 2^11 (complex128) / 2^12 (complex64) amplitudes
    int64_t mem_limit = 0;
    bool kernel_timing = false;
    bool dry_run = false;
    bool reg_kernel = true;
    bool tma = false;  // the bulk-copy staged persistent kernel measured slower than one CTA per tile
    bool test_stall = false;
    bool tc_blocks = false;    // complex64: fused blocks on the tensor cores
    int tc_threshold10 = 40;   // ... when their register-kernel cost exceeds this / 10 dense ops

    // committed plan (matches the slabs when device_valid)
    bool have_plan = false;
    PlanParams plan_pp;
    int plan_G = 0;
    bool plan_reg = true;  // reg_kernel when the plan was committed
    std::vector<SegPlan> plans;
    std::vector<std::vector<Bitset>> supps;
    std::vector<std::vector<qt_gate>> plan_gates;  // the gates each segment of the plan was planned from
    bool device_valid = false;
    bool state_stale = false;  // set by dry runs

    // introspection of the last update
    std::vector<Bitset> last_F, last_W;

    // Encoded, layout-planned ops of every pass of the last update's plan, by
    // segment and pass: a pass the next update plans again (same ops, same
    // tile) reuses them instead of being encoded and laid out anew.  Entries
    // depend only on the pass and on enc_pp / enc_reg (cleared when those
    // change); passes with tensor-core blocks are not kept.
    struct EncPass {
        bool valid = false;
        Pass ps;
        DevPass dp;  // the fields the layout planner and set_register_offsets fill
        std::vector<DevOp> ops;
    };
    std::vector<std::vector<EncPass>> enc;
    PlanParams enc_pp;
    bool enc_reg = false;

    // device
    bool device_ready = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void*> slabs;
    DevOp* d_ops = nullptr;
    size_t d_ops_cap = 0;
    uint32_t* d_wl = nullptr;
    size_t d_wl_cap = 0;
    float* d_blk = nullptr;  // operands B of the tensor-core blocks
    size_t d_blk_cap = 0;
    float* h_blk = nullptr;  // pinned staging
    size_t h_blk_cap = 0;
    DevOp* h_ops = nullptr;  // pinned staging
    size_t h_ops_cap = 0;
    uint32_t* h_wl = nullptr;
    size_t h_wl_cap = 0;
    double* d_norm_partials = nullptr;
    double* d_norm_out = nullptr;
    double* d_red = nullptr;   // reduction partial sums (fidelity, probabilities)
    size_t d_red_cap = 0;      // in doubles
    double* d_red_out = nullptr;
    size_t d_red_out_cap = 0;
    int norm_cap = 0;
    void* d_read = nullptr;
    size_t d_read_cap = 0;
    // qt_read_amplitudes_async: device snapshot of the converted amplitudes,
    // copied to the host on copy_stream while the circuit's stream goes on
    void* d_snap = nullptr;
    size_t d_snap_cap = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_snap = nullptr, ev_copy = nullptr;
    bool read_inflight = false;
    int* d_err = nullptr;  // set by a kernel whose bounded wait expired
    int* h_err = nullptr;  // pinned copy read after each update
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    std::vector<cudaEvent_t> ev_pool;

    std::string err;

    uint64_t namps() const { return uint64_t(1) << n; }
    uint32_t nparts() const { return uint32_t(1) << (n - p); }
    size_t state_bytes() const { return size_t(namps()) * bytes_per_amp(dtype); }
};

namespace {

qt_status fail(qt_circuit* c, qt_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

qt_status cuda_fail(qt_circuit* c, int e, const char* what) {
    return fail(c, QT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(cudaError_t(e)));
}

int lowest_qubit(const qt_gate& g) {
    int m = 1 << 30;
    for (int k = 0; k < g.ntarget; ++k) m = std::min(m, g.target[k]);
    for (int k = 0; k < g.ncontrol; ++k) m = std::min(m, g.control[k]);
    return m;
}

uint64_t level_qubits(const Level& L, qt_gate_id skip) {
    uint64_t m = 0;
    for (const Gate& g : L.gates)
        if (g.id != skip) m |= gate_qubit_mask(g.g);
    return m;
}

void insert_sorted(Level& L, const Gate& g) {
    int key = lowest_qubit(g.g);
    auto it = std::find_if(L.gates.begin(), L.gates.end(), [&](const Gate& x) { return lowest_qubit(x.g) > key; });
    L.gates.insert(it, g);
}

void free_device(qt_circuit* c) {
    if (!c->device_ready) return;
    cudaStreamSynchronize(c->stream);
    if (c->read_inflight) cudaEventSynchronize(c->ev_copy);
    c->read_inflight = false;
    cudaFree(c->d_snap);
    c->d_snap = nullptr;
    c->d_snap_cap = 0;
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->ev_snap) cudaEventDestroy(c->ev_snap);
    if (c->ev_copy) cudaEventDestroy(c->ev_copy);
    c->copy_stream = nullptr;
    c->ev_snap = c->ev_copy = nullptr;
    for (void* s : c->slabs) cudaFree(s);
    c->slabs.clear();
    cudaFree(c->d_ops);
    cudaFree(c->d_wl);
    cudaFreeHost(c->h_ops);
    cudaFreeHost(c->h_wl);
    cudaFree(c->d_blk);
    cudaFreeHost(c->h_blk);
    c->d_blk = nullptr;
    c->d_blk_cap = 0;
    c->h_blk = nullptr;
    c->h_blk_cap = 0;
    cudaFree(c->d_norm_partials);
    cudaFree(c->d_norm_out);
    cudaFree(c->d_red);
    cudaFree(c->d_red_out);
    cudaFree(c->d_read);
    cudaFree(c->d_err);
    cudaFreeHost(c->h_err);
    if (c->ev_begin) cudaEventDestroy(c->ev_begin);
    if (c->ev_end) cudaEventDestroy(c->ev_end);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    if (c->own_stream && c->stream) {
        cudaStreamDestroy(c->stream);
        c->stream = nullptr;
        c->own_stream = false;
    }
    // everything is reallocated by the next ensure_device()
    c->d_ops = nullptr;
    c->d_ops_cap = 0;
    c->d_wl = nullptr;
    c->d_wl_cap = 0;
    c->h_ops = nullptr;
    c->h_ops_cap = 0;
    c->h_wl = nullptr;
    c->h_wl_cap = 0;
    c->d_norm_partials = nullptr;
    c->d_norm_out = nullptr;
    c->norm_cap = 0;
    c->d_red = nullptr;
    c->d_red_cap = 0;
    c->d_red_out = nullptr;
    c->d_red_out_cap = 0;
    c->d_read = nullptr;
    c->d_read_cap = 0;
    c->d_err = nullptr;
    c->h_err = nullptr;
    c->ev_begin = c->ev_end = nullptr;
    c->device_ready = false;
    c->device_valid = false;
}

// Create the stream and slab 0 (|0...0>).
qt_status ensure_device(qt_circuit* c) {
    if (c->device_ready) return QT_OK;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(c, QT_ERR_CUDA, std::string("no CUDA device available: ") + cudaGetErrorString(e));
    if (c->mem_limit > 0 && int64_t(c->state_bytes()) > c->mem_limit)
        return fail(c, QT_ERR_OOM, "mem_limit below one state vector");
    if (!c->stream) {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamCreate");
        c->own_stream = true;
    }
    if ((e = cudaEventCreate(&c->ev_begin)) != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
    if ((e = cudaEventCreate(&c->ev_end)) != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
    void* s0 = nullptr;
    e = cudaMalloc(&s0, c->state_bytes());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QT_ERR_OOM, "cudaMalloc of the state vector failed");
    }
    c->slabs.push_back(s0);
    int rc = launch_init_zero_state(c->dtype, s0, c->namps(), c->stream);
    if (rc) return cuda_fail(c, rc, "init state");
    if ((e = cudaMalloc(reinterpret_cast<void**>(&c->d_err), sizeof(int))) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QT_ERR_OOM, "cudaMalloc of the error flag failed");
    }
    if ((e = cudaMallocHost(reinterpret_cast<void**>(&c->h_err), sizeof(int))) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QT_ERR_OOM, "cudaMallocHost of the error flag failed");
    }
    *c->h_err = 0;
    c->device_ready = true;
    c->device_valid = false;
    return QT_OK;
}

qt_status ensure_slabs(qt_circuit* c, size_t nslabs) {
    if (c->mem_limit > 0 && int64_t(nslabs * c->state_bytes()) > c->mem_limit)
        return fail(c, QT_ERR_OOM,
                    "checkpoints need " + std::to_string(nslabs) + " state vectors, above mem_limit");
    while (c->slabs.size() < nslabs) {
        void* s = nullptr;
        cudaError_t e = cudaMalloc(&s, c->state_bytes());
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, QT_ERR_OOM, "cudaMalloc of a checkpoint slab failed");
        }
        c->slabs.push_back(s);
    }
    return QT_OK;
}

template <class T>
qt_status grow_device(qt_circuit* c, T** d, size_t* cap, size_t need) {
    if (need <= *cap) return QT_OK;
    size_t ncap = std::max<size_t>(need, *cap * 2);
    cudaFree(*d);
    *d = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d), ncap * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QT_ERR_OOM, "cudaMalloc of a plan buffer failed");
    }
    *cap = ncap;
    return QT_OK;
}

template <class T>
qt_status grow_host(qt_circuit* c, T** h, size_t* cap, size_t need) {
    if (need <= *cap) return QT_OK;
    size_t ncap = std::max<size_t>(need, *cap * 2);
    cudaFreeHost(*h);
    *h = nullptr;
    *cap = 0;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(h), ncap * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QT_ERR_OOM, "cudaMallocHost of a staging buffer failed");
    }
    *cap = ncap;
    return QT_OK;
}

PlanParams make_params(const qt_circuit* c) {
    PlanParams pp;
    pp.n = c->n;
    pp.p = c->p;
    pp.lt = std::min(c->p, tile_low_default(c->dtype));
    pp.nh_max = std::max(0, std::min(c->tile_high, c->n - pp.lt));
    pp.fusion = c->fusion;
    pp.merge = c->merge;
    pp.tc_blocks = c->tc_blocks && c->dtype == QT_C64 && c->reg_kernel;
    pp.tc_threshold = c->tc_threshold10 / 10.0;
    return pp;
}

bool same_params(const PlanParams& a, const PlanParams& b) {
    return a.n == b.n && a.p == b.p && a.lt == b.lt && a.nh_max == b.nh_max && a.fusion == b.fusion &&
           a.merge == b.merge && a.tc_blocks == b.tc_blocks && a.tc_threshold == b.tc_threshold;
}

DevOp encode_op(int dtype, const Pass& ps, const HostOp& op, std::vector<float>* blkbuf = nullptr) {
    DevOp d;
    std::memset(&d, 0, sizeof d);
    auto loc = [&](int q) -> int {
        if (q < ps.lt) return q;
        for (int k = 0; k < ps.nh; ++k)
            if (ps.h[k] == q) return ps.lt + k;
        return -1;
    };
    if (op.kind == OP_BLOCK) {
        // tensor-core block: its tile bits, the other tile bits (rows), and
        // its operand B appended to the update's block buffer
        if (!blkbuf) throw std::logic_error("block op without a block buffer");
        const Block& b = ps.blocks.at(size_t(op.q0));
        d.kind = OP_BLOCK;
        d.b0 = d.b1 = d.gq = -1;
        BlockStage& bs = *reinterpret_cast<BlockStage*>(&d.m);
        uint32_t in = 0;
        for (int i = 0; i < 5; ++i) {
            bs.s[i] = int8_t(loc(b.q[i]));
            in |= 1u << bs.s[i];
        }
        int r = 0;
        for (int t = 0; t < ps.lt + ps.nh; ++t)
            if (!((in >> t) & 1u)) bs.rows[r++] = int8_t(t);
        if (r != 7) throw std::logic_error("block op needs a tile of 12 bits");
        bs.boff = int64_t(blkbuf->size() * sizeof(float));
        const size_t at = blkbuf->size();
        blkbuf->resize(at + kBlockBytes / sizeof(float));
        block_operand(b, blkbuf->data() + at);
        return d;
    }
    uint64_t tile_mask = (uint64_t(1) << ps.lt) - 1;
    for (int k = 0; k < ps.nh; ++k) tile_mask |= uint64_t(1) << ps.h[k];
    d.kind = op.kind;
    // Only X, SWAP and PHASE ops carry conditions (CNOT/CCX, CZ/CP lower to
    // them); the register kernel applies the other kinds unpredicated.
    if (op.cmask != 0 && op.kind != OP_X && op.kind != OP_SWAP && op.kind != OP_PHASE)
        throw std::logic_error("controlled op of a kind that takes no controls");
    d.cm_glob = op.cmask & ~tile_mask;
    std::vector<std::pair<int, int>> fixed;  // (tile-local position, value)
    for (int q = 0; q < 64; ++q)
        if (((op.cmask & tile_mask) >> q) & 1) fixed.push_back({loc(q), 1});
    d.b0 = op.q0 >= 0 ? loc(op.q0) : -1;
    d.gq = op.q0;
    d.b1 = -1;
    switch (op.kind) {
        case OP_DENSE: case OP_REAL: case OP_IREAL: case OP_X: case OP_ANTI:
            fixed.push_back({d.b0, 0});
            break;
        case OP_SWAP:
            d.b1 = loc(op.q1);
            fixed.push_back({d.b0, 1});
            fixed.push_back({d.b1, 0});
            break;
        case OP_PHASE: {
            const double re = op.m[0], im = op.m[1];
            d.sub = PH_GENERAL;
            if (re == -1.0 && im == 0.0) d.sub = PH_NEG;
            else if (re == 0.0 && im == 1.0) d.sub = PH_POS_I;
            else if (re == 0.0 && im == -1.0) d.sub = PH_NEG_I;
            break;
        }
        default: break;
    }
    // tile-local control mask (the register-layout planner splits it)
    d.cm_tile = 0;
    for (int q = 0; q < 64; ++q)
        if (((op.cmask & tile_mask) >> q) & 1) d.cm_tile |= 1u << loc(q);
    std::sort(fixed.begin(), fixed.end());
    d.nfix = uint8_t(fixed.size());
    d.fixval = 0;
    for (size_t k = 0; k < fixed.size(); ++k) {
        d.fixpos[k] = int8_t(fixed[k].first);
        if (fixed[k].second) d.fixval |= uint8_t(1u << k);
    }
    encode_matrix(dtype, op, &d);
    return d;
}

cudaEvent_t pool_event(qt_circuit* c, size_t i) {
    while (c->ev_pool.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[i];
}

// Levels per checkpoint segment.  With a checkpoint budget: the interval of
// the current plan while its slabs (one per segment plus the initial state)
// still fit, else the smallest interval whose slabs fit (a new interval
// makes the next update full).
int effective_interval(const qt_circuit* c) {
    if (c->ckpt_budget <= 0) return c->ckpt_interval;
    const int64_t L = int64_t(c->levels.size());
    const int64_t slabs = std::max<int64_t>(2, c->ckpt_budget / int64_t(c->state_bytes()));
    auto fits = [&](int64_t G) { return (L + G - 1) / G + 1 <= slabs; };
    if (c->have_plan && c->plan_G > 0 && fits(c->plan_G)) return c->plan_G;
    const int64_t G = std::max<int64_t>(1, (L + slabs - 2) / (slabs - 1));
    return int(std::min<int64_t>(G, 1 << 20));
}

// The gates of a segment compared field by field (angles bit for bit).
bool same_gates(const std::vector<qt_gate>& a, const std::vector<qt_gate>& b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i) {
        const qt_gate &x = a[i], &y = b[i];
        if (x.kind != y.kind || x.ntarget != y.ntarget || x.ncontrol != y.ncontrol) return false;
        for (int k = 0; k < x.ntarget && k < 2; ++k)
            if (x.target[k] != y.target[k]) return false;
        for (int k = 0; k < x.ncontrol && k < 2; ++k)
            if (x.control[k] != y.control[k]) return false;
        if (std::memcmp(x.theta, y.theta, sizeof x.theta) != 0) return false;
    }
    return true;
}

// The DevPass fields that plan_register_layout and set_register_offsets fill.
void copy_planned_fields(const DevPass& from, DevPass* to) {
    to->reg_kernel = from.reg_kernel;
    to->nreg = from.nreg;
    to->nwarp = from.nwarp;
    std::memcpy(to->layout, from.layout, sizeof to->layout);
    to->fin = from.fin;
    to->groups = from.groups;
    to->mma = from.mma;
    std::memcpy(to->rin, from.rin, sizeof to->rin);
    std::memcpy(to->rout, from.rout, sizeof to->rout);
}

qt_status do_update(qt_circuit* c, int force_full, qt_update_stats* stats) {
    auto t0 = std::chrono::steady_clock::now();
    qt_update_stats st;
    std::memset(&st, 0, sizeof st);
    st.gpu_ms = -1.0;
    st.pass_kernel_ms = -1.0;

    // ---- plan
    const PlanParams pp = make_params(c);
    const int G = effective_interval(c);
    const int L = int(c->levels.size());
    const int S = (L + G - 1) / G;
    std::vector<SegPlan> nplans(S);
    std::vector<std::vector<Bitset>> nsupps(S);
    const uint32_t nparts = c->nparts();
    int64_t ngates_total = 0;
    // a segment whose gates are those it was planned from last time (same
    // parameters) keeps its plan: plan_segment is a function of both
    std::vector<std::vector<qt_gate>> nseg_gates(S);
    const bool reuse = c->have_plan && same_params(pp, c->plan_pp);
    for (int s = 0; s < S; ++s) {
        std::vector<const qt_gate*> gl;
        const int l0 = s * G, l1 = std::min(L, (s + 1) * G);
        for (int l = l0; l < l1; ++l)
            for (const Gate& g : c->levels[l].gates) gl.push_back(&g.g);
        ngates_total += int64_t(gl.size());
        nseg_gates[s].reserve(gl.size());
        for (const qt_gate* g : gl) nseg_gates[s].push_back(*g);
        if (reuse && s < int(c->plans.size()) && s < int(c->plan_gates.size()) &&
            same_gates(nseg_gates[s], c->plan_gates[s])) {
            nplans[s] = c->plans[s];
            nsupps[s] = c->supps[s];
        } else {
            nplans[s] = plan_segment(gl, pp);
            for (const Pass& ps : nplans[s].passes) nsupps[s].push_back(pass_support(ps, nparts));
        }
        nplans[s].first_level = l0;
        nplans[s].nlevels = l1 - l0;
    }
    // a change of kernel family (register or shared-memory kernel) re-runs
    // everything, so the state always comes from the current options' kernels
    const bool params_changed =
        !c->have_plan || !same_params(pp, c->plan_pp) || G != c->plan_G || c->reg_kernel != c->plan_reg;
    bool full = force_full || params_changed || (!c->dry_run && !c->device_valid);

    // ---- device
    if (!c->dry_run) {
        qt_status rs = ensure_device(c);
        if (rs != QT_OK) return rs;
        rs = ensure_slabs(c, size_t(S) + 1);
        if (rs != QT_OK) return rs;
        if (!c->device_valid) full = true;
    }

    // ---- track and schedule
    std::vector<Launch> launches;
    if (!same_params(pp, c->enc_pp) || c->enc_reg != c->reg_kernel) c->enc.clear();
    std::vector<std::vector<qt_circuit::EncPass>> next_enc(S);
    // the cached encoding of pass i of segment s, if that pass is unchanged:
    // at the same index, or at the same distance from the segment's end
    auto cached = [&](int s, size_t i, const Pass& ps) -> qt_circuit::EncPass* {
        if (!ps.blocks.empty() || s >= int(c->enc.size())) return nullptr;
        std::vector<qt_circuit::EncPass>& old = c->enc[s];
        const size_t nnew = nplans[s].passes.size();
        for (size_t k : {i, i + old.size() - nnew}) {
            if (k < old.size() && old[k].valid && old[k].ps.same_as(ps)) return &old[k];
        }
        return nullptr;
    };
    std::vector<DevOp> hops;
    std::vector<uint32_t> hwl;
    std::vector<float> hblk;  // operands B of the tensor-core blocks
    std::vector<Bitset> lastF(S), lastW(S);
    uint64_t seg_amp_updates = 0;
    Bitset dirty_in;
    dirty_in.resize(nparts);
    const int old_S = c->have_plan ? int(c->plans.size()) : 0;
    for (int s = 0; s < S; ++s) {
        const SegPlan& np = nplans[s];
        const std::vector<Bitset>& sup = nsupps[s];
        Bitset F, W;
        F.resize(nparts);
        W.resize(nparts);
        if (full || s >= old_S) {
            F.fill();
            W.fill();
        } else {
            const SegPlan& op = c->plans[s];
            const std::vector<Bitset>& osup = c->supps[s];
            const size_t lo = op.passes.size(), ln = np.passes.size();
            size_t j = 0;
            while (j < lo && j < ln && op.passes[j].same_as(np.passes[j])) ++j;
            size_t k = 0;
            while (k < lo - j && k < ln - j && op.passes[lo - 1 - k].same_as(np.passes[ln - 1 - k])) ++k;
            const bool same_plan = (j == lo && j == ln);
            if (!(same_plan && !dirty_in.any())) {
                Bitset seeds;
                seeds.resize(nparts);
                for (size_t i = j; i < lo - k; ++i) seeds.or_with(osup[i]);
                for (size_t i = j; i < ln - k; ++i) seeds.or_with(sup[i]);
                Bitset D = dirty_in;
                for (size_t i = 0; i < ln; ++i) {
                    if (i == j) D.or_with(seeds);
                    close_forward(&D, np.passes[i], sup[i]);
                }
                if (j >= ln) D.or_with(seeds);
                F = D;
                W = F;
                close_all(&W, np.passes, sup);
            }
        }
        lastF[s] = F;
        lastW[s] = W;
        dirty_in = F;
        next_enc[s].resize(np.passes.size());
        if (!W.any()) {
            // nothing to run: keep the segment's cached encodings for later updates
            for (size_t i = 0; i < np.passes.size(); ++i) {
                if (qt_circuit::EncPass* e = cached(s, i, np.passes[i])) {
                    next_enc[s][i] = std::move(*e);
                    e->valid = false;
                }
            }
            continue;
        }
        st.segments_run += 1;
        {
            // every gate of the segment is (re)applied to the recomputed partitions W
            int64_t seg_gates = 0;
            for (const Pass& ps : np.passes) seg_gates += ps.ngates;
            seg_amp_updates += W.count() * (uint64_t(1) << c->p) * uint64_t(seg_gates);
        }
        if (np.passes.empty()) {
            Launch ln{};
            ln.kind = 1;
            ln.seg = s;
            ln.wl_offset = hwl.size();
            for (uint32_t q = 0; q < nparts; ++q)
                if (W.get(q)) hwl.push_back(q);
            ln.ngroups = uint32_t(hwl.size() - ln.wl_offset);
            ln.parts_processed = ln.ngroups;
            launches.push_back(ln);
            continue;
        }
        for (size_t i = 0; i < np.passes.size(); ++i) {
            const Pass& ps = np.passes[i];
            Launch ln{};
            ln.kind = 0;
            ln.seg = s;
            ln.pass_idx = int64_t(i);
            ln.out_of_place = (i == 0);
            ln.ngates = ps.ngates;
            // groups: members of W (first pass) or of W n supp (later passes)
            Bitset T = W;
            if (i > 0)
                for (size_t w = 0; w < T.w.size(); ++w) T.w[w] &= sup[i].w[w];
            if (!T.any()) continue;
            const uint32_t gcount_all = nparts >> __builtin_popcount(ps.M);
            ln.wl_offset = hwl.size();
            if (T.all()) {
                ln.null_worklist = true;
                ln.ngroups = gcount_all;
            } else {
                ln.null_worklist = false;
                Bitset mark;
                mark.resize(nparts);
                for (uint32_t q = 0; q < nparts; ++q) {
                    if (!T.get(q)) continue;
                    uint32_t g = q & ~ps.M;
                    if (!mark.get(g)) {
                        mark.set(g);
                        hwl.push_back(g);
                    }
                }
                ln.ngroups = uint32_t(hwl.size() - ln.wl_offset);
            }
            ln.parts_processed = uint64_t(ln.ngroups) << __builtin_popcount(ps.M);
            ln.alu_per_amp = 0.0;
            for (const HostOp& o : ps.ops) ln.alu_per_amp += op_alu_per_amp(c->dtype, o);
            ln.nblocks = int(ps.blocks.size());
            DevPass& dp = ln.dp;
            std::memset(&dp, 0, sizeof dp);
            dp.p = c->p;
            dp.lt = ps.lt;
            dp.nh = ps.nh;
            dp.nins = 0;
            for (int h = 0; h < ps.nh; ++h) {
                dp.h[h] = ps.h[h];
                if (ps.h[h] < c->p) dp.ins[dp.nins++] = ps.h[h];
            }
            dp.tpg_log2 = c->p - ps.lt - dp.nins;
            dp.nops = int32_t(ps.ops.size());
            dp.M = ps.M;
            dp.npart_log2 = c->n - c->p;
            dp.op_offset = int64_t(hops.size());
            std::vector<DevOp> pops;
            qt_circuit::EncPass* hit = cached(s, i, ps);
            if (hit) {
                pops = hit->ops;
                copy_planned_fields(hit->dp, &dp);
                next_enc[s][i] = std::move(*hit);
                hit->valid = false;
            } else {
                pops.reserve(ps.ops.size());
                for (const HostOp& o : ps.ops) pops.push_back(encode_op(c->dtype, ps, o, &hblk));
                if (c->reg_kernel) {
                    plan_register_layout(&dp, &pops, int(bytes_per_amp(c->dtype)), true, true, c->dtype == QT_C64);
                    if (dp.reg_kernel) set_register_offsets(&dp);
                }
                if (ps.blocks.empty()) next_enc[s][i] = qt_circuit::EncPass{true, ps, dp, pops};
            }
            dp.tma = (dp.reg_kernel && c->tma) ? 1 : 0;
            dp.test_stall = c->test_stall ? 1 : 0;
            dp.nops = int32_t(pops.size());
            hops.insert(hops.end(), pops.begin(), pops.end());
            launches.push_back(ln);
        }
    }

    c->enc.swap(next_enc);
    c->enc_pp = pp;
    c->enc_reg = c->reg_kernel;

    // ---- stats (plan side)
    st.segments_total = S;
    st.gates_total = int32_t(ngates_total);
    for (int s = 0; s < S; ++s) {
        st.passes_total += int32_t(nplans[s].passes.size());
        st.partition_passes_total += int64_t(nplans[s].passes.size()) * nparts;
    }
    const uint64_t part_amps = uint64_t(1) << c->p;
    const uint64_t bpa = bytes_per_amp(c->dtype);
    for (const Launch& ln : launches) {
        st.launches += 1;
        if (ln.kind == 0) {
            st.passes_run += 1;
            st.partition_passes_run += int64_t(ln.parts_processed);
            st.tensor_blocks += ln.nblocks;
        }
        st.hbm_bytes += 2 * bpa * ln.parts_processed * part_amps;
    }
    st.amp_updates = seg_amp_updates;
    st.clean_fraction =
        st.partition_passes_total ? 1.0 - double(st.partition_passes_run) / double(st.partition_passes_total) : 0.0;

    // ---- run
    if (!c->dry_run) {
        qt_status rs;
        if ((rs = grow_device(c, &c->d_ops, &c->d_ops_cap, std::max<size_t>(hops.size(), 1))) != QT_OK) return rs;
        if ((rs = grow_device(c, &c->d_wl, &c->d_wl_cap, std::max<size_t>(hwl.size(), 1))) != QT_OK) return rs;
        if ((rs = grow_host(c, &c->h_ops, &c->h_ops_cap, std::max<size_t>(hops.size(), 1))) != QT_OK) return rs;
        if ((rs = grow_host(c, &c->h_wl, &c->h_wl_cap, std::max<size_t>(hwl.size(), 1))) != QT_OK) return rs;
        if (!hblk.empty()) {
            if ((rs = grow_device(c, &c->d_blk, &c->d_blk_cap, hblk.size())) != QT_OK) return rs;
            if ((rs = grow_host(c, &c->h_blk, &c->h_blk_cap, hblk.size())) != QT_OK) return rs;
            std::memcpy(c->h_blk, hblk.data(), hblk.size() * sizeof(float));
        }
        st.h2d_bytes = hops.size() * sizeof(DevOp) + hwl.size() * sizeof(uint32_t) + hblk.size() * sizeof(float);
        if (!hops.empty()) std::memcpy(c->h_ops, hops.data(), hops.size() * sizeof(DevOp));
        if (!hwl.empty()) std::memcpy(c->h_wl, hwl.data(), hwl.size() * sizeof(uint32_t));
        cudaError_t e;
        c->device_valid = false;  // until the whole schedule has run
        if ((e = cudaEventRecord(c->ev_begin, c->stream)) != cudaSuccess) return cuda_fail(c, e, "event");
        if ((e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "error flag");
        if (!hops.empty() &&
            (e = cudaMemcpyAsync(c->d_ops, c->h_ops, hops.size() * sizeof(DevOp), cudaMemcpyHostToDevice,
                                 c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "upload ops");
        if (!hwl.empty() &&
            (e = cudaMemcpyAsync(c->d_wl, c->h_wl, hwl.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                 c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "upload worklists");
        if (!hblk.empty() &&
            (e = cudaMemcpyAsync(c->d_blk, c->h_blk, hblk.size() * sizeof(float), cudaMemcpyHostToDevice,
                                 c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "upload blocks");
        size_t evi = 0;
        for (const Launch& ln : launches) {
            void* src = c->slabs[ln.seg];
            void* dst = c->slabs[ln.seg + 1];
            int rc;
            if (ln.kind == 1) {
                rc = launch_copy_parts(c->dtype, dst, src, c->p, c->d_wl + ln.wl_offset, ln.ngroups, c->stream);
            } else {
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (c->kernel_timing) {
                    e0 = pool_event(c, evi++);
                    e1 = pool_event(c, evi++);
                    if (!e0 || !e1) return fail(c, QT_ERR_CUDA, "event pool");
                    cudaEventRecord(e0, c->stream);
                }
                DevPass dp = ln.dp;
                if (dp.mma) dp.blk = reinterpret_cast<const unsigned char*>(c->d_blk);
                rc = launch_pass(c->dtype, dst, ln.out_of_place ? src : dst, dp, c->d_ops,
                                 ln.null_worklist ? nullptr : c->d_wl + ln.wl_offset, ln.ngroups, c->d_err,
                                 c->stream);
                if (c->kernel_timing) cudaEventRecord(e1, c->stream);
            }
            if (rc) return cuda_fail(c, rc, "kernel launch");
        }
        if ((e = cudaEventRecord(c->ev_end, c->stream)) != cudaSuccess) return cuda_fail(c, e, "event");
        if ((e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "error flag");
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "update_state");
        if (*c->h_err != 0)
            return fail(c, QT_ERR_TIMEOUT, "a bounded device wait expired (bulk copy did not complete in 1 s)");
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->ev_begin, c->ev_end) == cudaSuccess) st.gpu_ms = ms;
        if (c->kernel_timing) {
            double tot = 0.0;
            size_t k = 0;
            for (const Launch& ln : launches) {
                if (ln.kind != 0) continue;
                float km = 0.0f;
                cudaEventElapsedTime(&km, c->ev_pool[k], c->ev_pool[k + 1]);
                k += 2;
                tot += km;
                st.pass_kernel_launches += 1;
                st.pass_kernel_bytes += 2 * bpa * ln.parts_processed * part_amps;
                st.pass_kernel_alu_ops += uint64_t(ln.alu_per_amp * double(ln.parts_processed * part_amps));
            }
            st.pass_kernel_ms = tot;
        }
        c->device_valid = true;
        c->state_stale = false;
    } else {
        c->device_valid = false;
        c->state_stale = true;
        // the slabs beyond the committed plan hold nothing useful now
    }

    // ---- commit
    c->plans = std::move(nplans);
    c->supps = std::move(nsupps);
    c->plan_gates = std::move(nseg_gates);
    c->plan_pp = pp;
    c->plan_G = G;
    c->plan_reg = c->reg_kernel;
    c->have_plan = true;
    c->last_F = std::move(lastF);
    c->last_W = std::move(lastW);
    c->pending = false;
    if (!c->dry_run && c->device_ready) {
        // release slabs the plan no longer uses
        while (c->slabs.size() > size_t(S) + 1) {
            cudaFree(c->slabs.back());
            c->slabs.pop_back();
        }
    }
    st.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = st;
    return QT_OK;
}

const void* final_state(const qt_circuit* c) { return c->slabs[c->have_plan ? c->plans.size() : 0]; }

qt_status check_readable(qt_circuit* c) {
    if (c->pending) return fail(c, QT_ERR_STALE, "edits are pending: call qt_update_state first");
    if (c->state_stale) return fail(c, QT_ERR_STALE, "the last update was a dry run: the state was not computed");
    qt_status rs = ensure_device(c);
    if (rs != QT_OK) return rs;
    if (c->have_plan && !c->device_valid && !c->plans.empty())
        return fail(c, QT_ERR_STALE,
                    "the state is not on the device (released, or a previous update failed): call qt_update_state");
    return QT_OK;
}

}  // namespace

// ------------------------------------------------ hooks for batched runs --
DevOp qt::encode_device_op(int dtype, const Pass& ps, const HostOp& op) { return encode_op(dtype, ps, op); }
DevOp qt::encode_device_op(int dtype, const Pass& ps, const HostOp& op, std::vector<float>* blkbuf) {
    return encode_op(dtype, ps, op, blkbuf);
}

void qt::circuit_plan_whole(const qt_circuit* c, std::vector<Pass>* passes, int* dtype, int* n) {
    PlanParams pp = make_params(c);
    pp.p = c->n;  // one partition: tiles may use every qubit, no coupling
    pp.tc_blocks = false;  // the batch kernel has no tensor-core blocks
    pp.lt = std::min(c->n, tile_low_default(c->dtype));
    pp.nh_max = std::max(0, std::min(c->tile_high, c->n - pp.lt));
    std::vector<const qt_gate*> gl;
    for (const Level& L : c->levels)
        for (const Gate& g : L.gates) gl.push_back(&g.g);
    SegPlan sp = plan_segment(gl, pp);
    *passes = std::move(sp.passes);
    *dtype = c->dtype;
    *n = c->n;
}

// ===================================================================== ABI ==
#define QT_GUARD_BEGIN try {
#define QT_GUARD_END(c)                                                    \
    }                                                                      \
    catch (const std::bad_alloc&) {                                        \
        return fail(c, QT_ERR_OOM, "host allocation failed");              \
    }                                                                      \
    catch (...) {                                                          \
        return fail(c, QT_ERR_ARG, "internal error (unexpected exception)"); \
    }

extern "C" {

qt_status qt_create(int32_t n_qubits, int32_t dtype, int32_t log2_partition, qt_circuit** out) {
    if (!out) {
        g_create_error = "out is NULL";
        return QT_ERR_ARG;
    }
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > kMaxQubits) {
        g_create_error = "n_qubits must be in [1, 34]";
        return QT_ERR_ARG;
    }
    if (dtype != QT_C128 && dtype != QT_C64 && dtype != QT_C128_DF) {
        g_create_error = "unknown dtype";
        return QT_ERR_ARG;
    }
    if (log2_partition < 0 || log2_partition > n_qubits || n_qubits - log2_partition > 30) {
        g_create_error = "log2_partition must be in [max(0, n-30), n]";
        return QT_ERR_ARG;
    }
    try {
        qt_circuit* c = new qt_circuit();
        c->n = n_qubits;
        c->dtype = dtype;
        c->p = log2_partition;
        *out = c;
        return QT_OK;
    } catch (...) {
        g_create_error = "host allocation failed";
        return QT_ERR_OOM;
    }
}

qt_status qt_destroy(qt_circuit* c) {
    if (!c) return QT_OK;
    free_device(c);
    delete c;
    return QT_OK;
}

qt_status qt_num_levels(const qt_circuit* c, int32_t* out) {
    if (!c || !out) return QT_ERR_ARG;
    *out = int32_t(c->levels.size());
    return QT_OK;
}

qt_status qt_num_gates(const qt_circuit* c, int64_t* out) {
    if (!c || !out) return QT_ERR_ARG;
    int64_t k = 0;
    for (const Level& L : c->levels) k += int64_t(L.gates.size());
    *out = k;
    return QT_OK;
}

qt_status qt_insert_level(qt_circuit* c, int32_t pos) {
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    if (pos < 0 || pos > int32_t(c->levels.size())) return fail(c, QT_ERR_RANGE, "level position out of range");
    c->levels.insert(c->levels.begin() + pos, Level());
    c->pending = true;
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_remove_level(qt_circuit* c, int32_t pos) {
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    if (pos < 0 || pos >= int32_t(c->levels.size())) return fail(c, QT_ERR_RANGE, "level out of range");
    c->levels.erase(c->levels.begin() + pos);
    c->pending = true;
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_insert_gate(qt_circuit* c, int32_t level, const qt_gate* g, qt_gate_id* out) {
    if (!c) return QT_ERR_ARG;
    if (!g) return fail(c, QT_ERR_ARG, "gate is NULL");
    QT_GUARD_BEGIN
    std::string err;
    if (!check_gate(*g, c->n, &err)) return fail(c, QT_ERR_ARG, err);
    if (level < 0 || level >= int32_t(c->levels.size())) return fail(c, QT_ERR_RANGE, "level out of range");
    Level& L = c->levels[level];
    if (level_qubits(L, 0) & gate_qubit_mask(*g))
        return fail(c, QT_ERR_CONFLICT, "gate shares a qubit with a gate of level " + std::to_string(level));
    Gate ng;
    ng.g = *g;
    ng.id = c->next_id++;
    insert_sorted(L, ng);
    c->pending = true;
    if (out) *out = ng.id;
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_remove_gate(qt_circuit* c, int32_t level, qt_gate_id id) {
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    if (level < 0 || level >= int32_t(c->levels.size())) return fail(c, QT_ERR_RANGE, "level out of range");
    Level& L = c->levels[level];
    auto it = std::find_if(L.gates.begin(), L.gates.end(), [&](const Gate& x) { return x.id == id; });
    if (it == L.gates.end()) return fail(c, QT_ERR_NOT_FOUND, "no gate with that id in that level");
    L.gates.erase(it);
    c->pending = true;
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_replace_gate(qt_circuit* c, int32_t level, qt_gate_id id, const qt_gate* g, qt_gate_id* out) {
    if (!c) return QT_ERR_ARG;
    if (!g) return fail(c, QT_ERR_ARG, "gate is NULL");
    QT_GUARD_BEGIN
    std::string err;
    if (!check_gate(*g, c->n, &err)) return fail(c, QT_ERR_ARG, err);
    if (level < 0 || level >= int32_t(c->levels.size())) return fail(c, QT_ERR_RANGE, "level out of range");
    Level& L = c->levels[level];
    auto it = std::find_if(L.gates.begin(), L.gates.end(), [&](const Gate& x) { return x.id == id; });
    if (it == L.gates.end()) return fail(c, QT_ERR_NOT_FOUND, "no gate with that id in that level");
    if (level_qubits(L, id) & gate_qubit_mask(*g))
        return fail(c, QT_ERR_CONFLICT, "replacement shares a qubit with another gate of the level");
    L.gates.erase(it);
    Gate ng;
    ng.g = *g;
    ng.id = c->next_id++;
    insert_sorted(L, ng);
    c->pending = true;
    if (out) *out = ng.id;
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_update_state(qt_circuit* c, int32_t force_full, qt_update_stats* stats) {
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    return do_update(c, force_full, stats);
    QT_GUARD_END(c)
}

qt_status qt_read_amplitudes(const qt_circuit* cc, uint64_t first, uint64_t count, void* host_dst) {
    qt_circuit* c = const_cast<qt_circuit*>(cc);
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    if (count && !host_dst) return fail(c, QT_ERR_ARG, "host_dst is NULL");
    if (first > c->namps() || count > c->namps() - first) return fail(c, QT_ERR_RANGE, "amplitude range");
    qt_status rs = check_readable(c);
    if (rs != QT_OK) return rs;
    if (count == 0) return QT_OK;
    const void* src = final_state(c);
    cudaError_t e;
    if (c->dtype != QT_C128_DF) {
        const size_t b = bytes_per_amp(c->dtype);
        e = cudaMemcpyAsync(host_dst, static_cast<const char*>(src) + first * b, count * b, cudaMemcpyDeviceToHost,
                            c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "read amplitudes");
    } else {
        const uint64_t chunk = uint64_t(1) << 22;  // amplitudes per staging round (64 MiB)
        const size_t need = size_t(std::min(count, chunk)) * 16;
        if (c->d_read_cap < need) {
            cudaFree(c->d_read);
            c->d_read = nullptr;
            c->d_read_cap = 0;
            if ((e = cudaMalloc(&c->d_read, need)) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, QT_ERR_OOM, "staging buffer");
            }
            c->d_read_cap = need;
        }
        for (uint64_t off = 0; off < count; off += chunk) {
            const uint64_t m = std::min(chunk, count - off);
            int rc = launch_read_convert(c->dtype, c->d_read, src, first + off, m, c->stream);
            if (rc) return cuda_fail(c, rc, "convert");
            e = cudaMemcpyAsync(static_cast<char*>(host_dst) + off * 16, c->d_read, m * 16, cudaMemcpyDeviceToHost,
                                c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "read amplitudes");
        }
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "read amplitudes");
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_read_amplitudes_async(qt_circuit* c, uint64_t first, uint64_t count, void* host_dst) {
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    if (count && !host_dst) return fail(c, QT_ERR_ARG, "host_dst is NULL");
    if (first > c->namps() || count > c->namps() - first) return fail(c, QT_ERR_RANGE, "amplitude range");
    qt_status rs = check_readable(c);
    if (rs != QT_OK) return rs;
    cudaError_t e;
    if (!c->copy_stream) {
        if ((e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "cudaStreamCreate");
        if ((e = cudaEventCreateWithFlags(&c->ev_snap, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "cudaEventCreate");
    }
    if (count == 0) return QT_OK;
    const size_t ob = c->dtype == QT_C64 ? 8 : 16;  // output bytes per amplitude
    const size_t need = size_t(count) * ob;
    // the snapshot buffer is free once the previous read's copy has finished
    if (c->read_inflight && (e = cudaStreamWaitEvent(c->stream, c->ev_copy, 0)) != cudaSuccess)
        return cuda_fail(c, e, "read amplitudes");
    if (c->d_snap_cap < need) {
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "read amplitudes");
        cudaFree(c->d_snap);
        c->d_snap = nullptr;
        c->d_snap_cap = 0;
        if ((e = cudaMalloc(&c->d_snap, need)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, QT_ERR_OOM, "snapshot buffer");
        }
        c->d_snap_cap = need;
    }
    int rc = launch_read_convert(c->dtype, c->d_snap, final_state(c), first, count, c->stream);
    if (rc) return cuda_fail(c, rc, "read amplitudes");
    if ((e = cudaEventRecord(c->ev_snap, c->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(c->copy_stream, c->ev_snap, 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(host_dst, c->d_snap, need, cudaMemcpyDeviceToHost, c->copy_stream)) != cudaSuccess ||
        (e = cudaEventRecord(c->ev_copy, c->copy_stream)) != cudaSuccess)
        return cuda_fail(c, e, "read amplitudes");
    c->read_inflight = true;
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_read_wait(qt_circuit* c) {
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    if (!c->read_inflight) return QT_OK;
    c->read_inflight = false;
    cudaError_t e = cudaEventSynchronize(c->ev_copy);
    if (e != cudaSuccess) return cuda_fail(c, e, "read amplitudes");
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_read_amplitudes_device(const qt_circuit* cc, uint64_t first, uint64_t count, void* device_dst) {
    qt_circuit* c = const_cast<qt_circuit*>(cc);
    if (!c) return QT_ERR_ARG;
    QT_GUARD_BEGIN
    if (count && !device_dst) return fail(c, QT_ERR_ARG, "device_dst is NULL");
    if (first > c->namps() || count > c->namps() - first) return fail(c, QT_ERR_RANGE, "amplitude range");
    qt_status rs = check_readable(c);
    if (rs != QT_OK) return rs;
    int rc = launch_read_convert(c->dtype, device_dst, final_state(c), first, count, c->stream);
    if (rc) return cuda_fail(c, rc, "read amplitudes");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read amplitudes");
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_fidelity(const qt_circuit* ca, const qt_circuit* cb, double* out) {
    qt_circuit* a = const_cast<qt_circuit*>(ca);
    qt_circuit* b = const_cast<qt_circuit*>(cb);
    if (!a) return QT_ERR_ARG;
    if (!b || !out) return fail(a, QT_ERR_ARG, "b and out must not be NULL");
    QT_GUARD_BEGIN
    if (a->n != b->n) return fail(a, QT_ERR_ARG, "the two circuits have different qubit counts");
    qt_status rs = check_readable(a);
    if (rs != QT_OK) return rs;
    rs = check_readable(b);
    if (rs != QT_OK) return fail(a, rs, std::string("second circuit: ") + b->err);
    cudaError_t e;
    if (b->stream != a->stream && (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return cuda_fail(a, e, "fidelity");
    const int nb = reduce_blocks(a->namps());
    if ((rs = grow_device(a, &a->d_red, &a->d_red_cap, size_t(4) * nb)) != QT_OK) return rs;
    if ((rs = grow_device(a, &a->d_red_out, &a->d_red_out_cap, 4)) != QT_OK) return rs;
    int rc = launch_fidelity(a->dtype, final_state(a), b->dtype, final_state(b), a->namps(), a->d_red, nb,
                             a->d_red_out, a->stream);
    if (rc) return cuda_fail(a, rc, "fidelity");
    double h[4];
    if ((e = cudaMemcpyAsync(h, a->d_red_out, sizeof h, cudaMemcpyDeviceToHost, a->stream)) != cudaSuccess)
        return cuda_fail(a, e, "fidelity");
    if ((e = cudaStreamSynchronize(a->stream)) != cudaSuccess) return cuda_fail(a, e, "fidelity");
    if (!(h[2] > 0.0) || !(h[3] > 0.0)) return fail(a, QT_ERR_ARG, "a state has zero norm");
    *out = (h[0] * h[0] + h[1] * h[1]) / (h[2] * h[3]);
    return QT_OK;
    QT_GUARD_END(a)
}

qt_status qt_max_abs_diff(const qt_circuit* ca, const qt_circuit* cb, double* out) {
    qt_circuit* a = const_cast<qt_circuit*>(ca);
    qt_circuit* b = const_cast<qt_circuit*>(cb);
    if (!a) return QT_ERR_ARG;
    if (!b || !out) return fail(a, QT_ERR_ARG, "b and out must not be NULL");
    QT_GUARD_BEGIN
    if (a->n != b->n) return fail(a, QT_ERR_ARG, "the two circuits have different qubit counts");
    qt_status rs = check_readable(a);
    if (rs != QT_OK) return rs;
    rs = check_readable(b);
    if (rs != QT_OK) return fail(a, rs, std::string("second circuit: ") + b->err);
    cudaError_t e;
    if (b->stream != a->stream && (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return cuda_fail(a, e, "max_abs_diff");
    const int nb = reduce_blocks(a->namps());
    if ((rs = grow_device(a, &a->d_red, &a->d_red_cap, size_t(nb))) != QT_OK) return rs;
    if ((rs = grow_device(a, &a->d_red_out, &a->d_red_out_cap, 4)) != QT_OK) return rs;
    int rc = launch_max_sq_diff(a->dtype, final_state(a), b->dtype, final_state(b), a->namps(), a->d_red, nb,
                                a->d_red_out, a->stream);
    if (rc) return cuda_fail(a, rc, "max_abs_diff");
    double h = 0.0;
    if ((e = cudaMemcpyAsync(&h, a->d_red_out, sizeof h, cudaMemcpyDeviceToHost, a->stream)) != cudaSuccess)
        return cuda_fail(a, e, "max_abs_diff");
    if ((e = cudaStreamSynchronize(a->stream)) != cudaSuccess) return cuda_fail(a, e, "max_abs_diff");
    *out = std::sqrt(h);
    return QT_OK;
    QT_GUARD_END(a)
}

qt_status qt_probabilities(const qt_circuit* cc, int32_t k, const int32_t* qubits, double* out) {
    qt_circuit* c = const_cast<qt_circuit*>(cc);
    if (!c) return QT_ERR_ARG;
    if (!out || (k > 0 && !qubits)) return fail(c, QT_ERR_ARG, "NULL argument");
    QT_GUARD_BEGIN
    if (k < 0 || k > 10) return fail(c, QT_ERR_ARG, "k must be in [0, 10]");
    QubitList ql;
    ql.k = k;
    uint64_t seen = 0;
    for (int j = 0; j < k; ++j) {
        if (qubits[j] < 0 || qubits[j] >= c->n || ((seen >> qubits[j]) & 1))
            return fail(c, QT_ERR_ARG, "qubits must be distinct and in [0, n)");
        seen |= uint64_t(1) << qubits[j];
        ql.q[j] = qubits[j];
    }
    qt_status rs = check_readable(c);
    if (rs != QT_OK) return rs;
    const int nb = reduce_blocks(c->namps());
    const size_t nbins = size_t(1) << k;
    if ((rs = grow_device(c, &c->d_red, &c->d_red_cap, nbins * nb)) != QT_OK) return rs;
    if ((rs = grow_device(c, &c->d_red_out, &c->d_red_out_cap, nbins)) != QT_OK) return rs;
    int rc = launch_probabilities(c->dtype, final_state(c), c->namps(), ql, c->d_red, nb, c->d_red_out, c->stream);
    if (rc) return cuda_fail(c, rc, "probabilities");
    cudaError_t e = cudaMemcpyAsync(out, c->d_red_out, nbins * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "probabilities");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "probabilities");
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_norm(const qt_circuit* cc, double* out) {
    qt_circuit* c = const_cast<qt_circuit*>(cc);
    if (!c) return QT_ERR_ARG;
    if (!out) return fail(c, QT_ERR_ARG, "out is NULL");
    QT_GUARD_BEGIN
    qt_status rs = check_readable(c);
    if (rs != QT_OK) return rs;
    const int np = norm_partials_needed(c->namps());
    cudaError_t e;
    if (c->norm_cap < np) {
        cudaFree(c->d_norm_partials);
        c->d_norm_partials = nullptr;
        c->norm_cap = 0;
        if ((e = cudaMalloc(&c->d_norm_partials, sizeof(double) * np)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, QT_ERR_OOM, "norm scratch");
        }
        c->norm_cap = np;
    }
    if (!c->d_norm_out && (e = cudaMalloc(&c->d_norm_out, sizeof(double))) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QT_ERR_OOM, "norm scratch");
    }
    int rc = launch_norm(c->dtype, final_state(c), c->namps(), c->d_norm_partials, np, c->d_norm_out, c->stream);
    if (rc) return cuda_fail(c, rc, "norm");
    e = cudaMemcpyAsync(out, c->d_norm_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "norm");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "norm");
    return QT_OK;
    QT_GUARD_END(c)
}

qt_status qt_set_option(qt_circuit* c, const char* key, int64_t value) {
    if (!c) return QT_ERR_ARG;
    if (!key) return fail(c, QT_ERR_ARG, "key is NULL");
    std::string k(key);
    if (k == "ckpt_interval") {
        if (value < 1 || value > (1 << 20)) return fail(c, QT_ERR_ARG, "ckpt_interval must be >= 1");
        c->ckpt_interval = int(value);
    } else if (k == "ckpt_budget") {
        if (value < 0) return fail(c, QT_ERR_ARG, "ckpt_budget must be >= 0");
        c->ckpt_budget = value;
    } else if (k == "fusion") {
        c->fusion = value != 0;
    } else if (k == "merge") {
        c->merge = value != 0;
    } else if (k == "tile_high") {
        if (value < 0 || value > kMaxTileHigh) return fail(c, QT_ERR_ARG, "tile_high must be in [0, 7]");
        if (tile_low_default(c->dtype) + value > (c->dtype == QT_C64 ? 13 : 12))
            return fail(c, QT_ERR_ARG, "tile too large for shared memory");
        c->tile_high = int(value);
    } else if (k == "mem_limit") {
        if (value < 0) return fail(c, QT_ERR_ARG, "mem_limit must be >= 0");
        c->mem_limit = value;
    } else if (k == "kernel_timing") {
        c->kernel_timing = value != 0;
    } else if (k == "tma") {
        c->tma = value != 0;
    } else if (k == "test_stall_staging") {
        c->test_stall = value != 0;
    } else if (k == "reg_kernel") {
        c->reg_kernel = value != 0;
    } else if (k == "tc_blocks") {
        c->tc_blocks = value != 0;
    } else if (k == "tc_threshold") {
        if (value < 0 || value > 1000) return fail(c, QT_ERR_ARG, "tc_threshold must be in [0, 1000]");
        c->tc_threshold10 = int(value);
    } else if (k == "dry_run") {
        c->dry_run = value != 0;
    } else {
        return fail(c, QT_ERR_ARG, "unknown option " + k);
    }
    return QT_OK;
}

qt_status qt_set_stream(qt_circuit* c, void* cuda_stream) {
    if (!c) return QT_ERR_ARG;
    if (c->device_ready) cudaStreamSynchronize(c->stream);
    if (c->own_stream && c->stream) {
        cudaStreamDestroy(c->stream);
        c->own_stream = false;
    }
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!c->stream && c->device_ready) {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(c, QT_ERR_CUDA, "cudaStreamCreate");
        c->own_stream = true;
    }
    return QT_OK;
}

qt_status qt_num_segments(const qt_circuit* c, int32_t* out) {
    if (!c || !out) return QT_ERR_ARG;
    *out = c->have_plan ? int32_t(c->plans.size()) : 0;
    return QT_OK;
}

qt_status qt_segment_info(const qt_circuit* cc, int32_t seg, int32_t* first_level, int32_t* nlevels,
                          int32_t* npasses, uint8_t* dirty_out, uint8_t* worklist_out) {
    qt_circuit* c = const_cast<qt_circuit*>(cc);
    if (!c) return QT_ERR_ARG;
    if (!c->have_plan || seg < 0 || seg >= int32_t(c->plans.size()))
        return fail(c, QT_ERR_RANGE, "segment out of range");
    const SegPlan& sp = c->plans[seg];
    if (first_level) *first_level = sp.first_level;
    if (nlevels) *nlevels = sp.nlevels;
    if (npasses) *npasses = int32_t(sp.passes.size());
    const uint32_t np = c->nparts();
    for (uint32_t q = 0; q < np; ++q) {
        if (dirty_out) dirty_out[q] = c->last_F[seg].get(q) ? 1 : 0;
        if (worklist_out) worklist_out[q] = c->last_W[seg].get(q) ? 1 : 0;
    }
    return QT_OK;
}

qt_status qt_segment_touched(const qt_circuit* cc, int32_t seg, uint8_t* touched_out) {
    qt_circuit* c = const_cast<qt_circuit*>(cc);
    if (!c || !touched_out) return QT_ERR_ARG;
    if (!c->have_plan || seg < 0 || seg >= int32_t(c->supps.size()))
        return fail(c, QT_ERR_RANGE, "segment out of range");
    const uint32_t np = c->nparts();
    Bitset U;
    U.resize(np);
    for (const Bitset& b : c->supps[seg]) U.or_with(b);
    for (uint32_t q = 0; q < np; ++q) touched_out[q] = U.get(q) ? 1 : 0;
    return QT_OK;
}

const char* qt_last_error(const qt_circuit* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

qt_status qt_release_device(qt_circuit* c) {
    if (!c) return QT_ERR_ARG;
    free_device(c);
    return QT_OK;
}

qt_status qt_device_bytes(const qt_circuit* c, int64_t* out) {
    if (!c || !out) return QT_ERR_ARG;
    *out = int64_t(qt::circuit_device_bytes(c));
    return QT_OK;
}

}  // extern "C"

// -------------------------------------------- hooks for the serving loop --
size_t qt::circuit_device_bytes(const qt_circuit* c) {
    return c->device_ready ? c->slabs.size() * c->state_bytes() : 0;
}

size_t qt::circuit_state_bytes(const qt_circuit* c) { return c->state_bytes(); }

size_t qt::circuit_device_need(const qt_circuit* c) {
    const size_t L = c->levels.size();
    const size_t G = size_t(effective_interval(c));
    const size_t S = (L + G - 1) / G;
    return (S + 2) * c->state_bytes();  // checkpoints, and a level's worth of slack for inserted levels
}

void qt::circuit_release_device(qt_circuit* c) { free_device(c); }

extern "C" {

}  // extern "C"
