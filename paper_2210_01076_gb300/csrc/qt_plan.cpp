// qt_plan.cpp -- host side of the hot path: gate matrices and classification,
// canonical order, tile fusion of a segment into passes, and the partition
// support / coupling sets used by the dirty-partition tracker.
//
// qTask references: gate set, Table 1 and Section III-A; matrices, Section
// II-A; non-superposition (swap and scale) versus superposition (matrix)
// gates, Section III-C; parallel gates of a net may be ordered arbitrarily,
// Section II-A; partitions of consecutive blocks, Section III-C; frontiers and
// reachable partitions, Section III-E.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "qt_internal.h"

namespace qt {

using cd = std::complex<double>;

namespace {

struct M2 {
    cd a[4];  // row-major 2x2
};

M2 mul(const M2& x, const M2& y) {  // x * y
    M2 r;
    r.a[0] = x.a[0] * y.a[0] + x.a[1] * y.a[2];
    r.a[1] = x.a[0] * y.a[1] + x.a[1] * y.a[3];
    r.a[2] = x.a[2] * y.a[0] + x.a[3] * y.a[2];
    r.a[3] = x.a[2] * y.a[1] + x.a[3] * y.a[3];
    return r;
}

void put(double* m, int k, cd v) {
    m[2 * k] = v.real();
    m[2 * k + 1] = v.imag();
}
cd get(const double* m, int k) { return cd(m[2 * k], m[2 * k + 1]); }

// Base 2x2 matrix of a one-target kind (for CNOT/CCX the X, for CZ the Z,
// for CP the phase diag(1, e^{i theta})).
bool base_matrix(const qt_gate& g, M2* U) {
    const double t = g.theta[0];
    const double c = std::cos(t / 2.0), s = std::sin(t / 2.0);
    const double r2 = 1.0 / std::sqrt(2.0);
    const cd I(0.0, 1.0);
    cd* a = U->a;
    a[0] = a[1] = a[2] = a[3] = 0.0;
    switch (g.kind) {
        case QT_H: a[0] = r2; a[1] = r2; a[2] = r2; a[3] = -r2; break;
        case QT_X: case QT_CNOT: case QT_CCX: a[1] = 1.0; a[2] = 1.0; break;
        case QT_Y: a[1] = -I; a[2] = I; break;
        case QT_Z: case QT_CZ: a[0] = 1.0; a[3] = -1.0; break;
        case QT_S: a[0] = 1.0; a[3] = I; break;
        case QT_SDG: a[0] = 1.0; a[3] = -I; break;
        case QT_T: a[0] = 1.0; a[3] = std::polar(1.0, M_PI / 4.0); break;
        case QT_TDG: a[0] = 1.0; a[3] = std::polar(1.0, -M_PI / 4.0); break;
        case QT_RX: a[0] = c; a[1] = -I * s; a[2] = -I * s; a[3] = c; break;
        case QT_RY: a[0] = c; a[1] = -s; a[2] = s; a[3] = c; break;
        case QT_RZ: a[0] = std::polar(1.0, -t / 2.0); a[3] = std::polar(1.0, t / 2.0); break;
        case QT_U3: {
            const double p = g.theta[1], l = g.theta[2];
            a[0] = c;
            a[1] = -std::polar(1.0, l) * s;
            a[2] = std::polar(1.0, p) * s;
            a[3] = std::polar(1.0, p + l) * c;
            break;
        }
        case QT_CP: a[0] = 1.0; a[3] = std::polar(1.0, t); break;
        default: return false;
    }
    return true;
}

// Classify a 2x2 by its exact structure (never by angle): diagonal,
// anti-diagonal, real, or general.  The paper's swap/scale versus matrix
// distinction (Section III-C) becomes the kernel specialisation.
HostOp classify(const M2& U, int q, uint64_t cmask, int ngates) {
    HostOp op;
    op.q0 = q;
    op.cmask = cmask;
    op.ngates = ngates;
    const cd *a = U.a;
    if (a[1] == 0.0 && a[2] == 0.0) {
        if (a[0] == 1.0) {
            op.kind = OP_PHASE;
            op.cmask |= uint64_t(1) << q;
            put(op.m, 0, a[3]);
        } else if (a[3] == 1.0) {
            // diag(d0, 1): a phase on the 0 value of q; keep it a DIAG.
            op.kind = OP_DIAG;
            put(op.m, 0, a[0]);
            put(op.m, 1, a[3]);
        } else {
            op.kind = OP_DIAG;
            put(op.m, 0, a[0]);
            put(op.m, 1, a[3]);
        }
        return op;
    }
    if (a[0] == 0.0 && a[3] == 0.0) {
        if (a[1] == 1.0 && a[2] == 1.0) {
            op.kind = OP_X;
        } else {
            op.kind = OP_ANTI;
            put(op.m, 0, a[1]);
            put(op.m, 1, a[2]);
        }
        return op;
    }
    bool real = true;
    for (int k = 0; k < 4; ++k) real = real && a[k].imag() == 0.0;
    // real diagonal, imaginary off-diagonal (RX): as cheap as a real 2x2
    const bool ireal = a[0].imag() == 0.0 && a[3].imag() == 0.0 && a[1].real() == 0.0 && a[2].real() == 0.0;
    op.kind = real ? OP_REAL : ireal ? OP_IREAL : OP_DENSE;
    for (int k = 0; k < 4; ++k) put(op.m, k, a[k]);
    return op;
}

bool op_matrix(const HostOp& op, M2* U) {
    cd* a = U->a;
    a[0] = a[1] = a[2] = a[3] = 0.0;
    switch (op.kind) {
        case OP_DENSE: case OP_REAL: case OP_IREAL:
            for (int k = 0; k < 4; ++k) a[k] = get(op.m, k);
            return true;
        case OP_DIAG: a[0] = get(op.m, 0); a[3] = get(op.m, 1); return true;
        case OP_PHASE: a[0] = 1.0; a[3] = get(op.m, 0); return true;
        case OP_X: a[1] = 1.0; a[2] = 1.0; return true;
        case OP_ANTI: a[1] = get(op.m, 0); a[2] = get(op.m, 1); return true;
        default: return false;
    }
}

// An op on one qubit with no other condition: mergeable into its neighbours.
bool single_qubit(const HostOp& op) {
    if (op.kind == OP_SWAP) return false;
    if (op.kind == OP_PHASE) return op.cmask == (uint64_t(1) << op.q0);
    return op.cmask == 0;
}

bool is_diagonal(const HostOp& op) { return op.kind == OP_DIAG || op.kind == OP_PHASE; }

uint64_t op_qubits(const HostOp& op) {
    uint64_t m = op.cmask;
    if (op.q0 >= 0) m |= uint64_t(1) << op.q0;
    if (op.q1 >= 0) m |= uint64_t(1) << op.q1;
    return m;
}

int popcount64(uint64_t x) { return __builtin_popcountll(x); }

// Instructions per amplitude of an op in float-float (the costliest
// arithmetic; the binary32 and binary64 kernels have the same proportions): a
// complex 2x2 is two 4-term dot products per amplitude, a real 2x2, a
// diagonal, an anti-diagonal or a general phase two 2-term ones (a phase runs
// predicated over all amplitudes of a thread), exact phases (-1, +-i) and
// permutations only move data.
int op_cost(const HostOp& op) {
    switch (op.kind) {
        case OP_DENSE: return 86;
        case OP_REAL: case OP_IREAL: case OP_DIAG: case OP_ANTI: return 38;
        case OP_PHASE: {
            const bool exact = (op.m[0] == -1.0 && op.m[1] == 0.0) || (op.m[0] == 0.0 && std::fabs(op.m[1]) == 1.0);
            return exact ? 4 : 38;
        }
        default: return 1;
    }
}

}  // namespace

uint64_t gate_qubit_mask(const qt_gate& g) {
    uint64_t m = 0;
    for (int k = 0; k < g.ntarget; ++k) m |= uint64_t(1) << g.target[k];
    for (int k = 0; k < g.ncontrol; ++k) m |= uint64_t(1) << g.control[k];
    return m;
}

bool check_gate(const qt_gate& g, int n, std::string* err) {
    static const int nt[QT_NUM_KINDS] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 1, 1};
    static const int nc[QT_NUM_KINDS] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0, 2, 1};
    if (g.kind < 0 || g.kind >= QT_NUM_KINDS) {
        *err = "unknown gate kind " + std::to_string(g.kind);
        return false;
    }
    if (g.ntarget != nt[g.kind] || g.ncontrol != nc[g.kind]) {
        *err = "wrong number of targets/controls for kind " + std::to_string(g.kind);
        return false;
    }
    uint64_t seen = 0;
    for (int k = 0; k < g.ntarget + g.ncontrol; ++k) {
        int q = k < g.ntarget ? g.target[k] : g.control[k - g.ntarget];
        if (q < 0 || q >= n) {
            *err = "qubit " + std::to_string(q) + " out of range";
            return false;
        }
        if ((seen >> q) & 1) {
            *err = "qubit " + std::to_string(q) + " used twice by one gate";
            return false;
        }
        seen |= uint64_t(1) << q;
    }
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(g.theta[k])) {
            *err = "non-finite angle";
            return false;
        }
    return true;
}

bool lower_gate(const qt_gate& g, int n, std::vector<HostOp>* out, std::string* err) {
    if (!check_gate(g, n, err)) return false;
    if (g.kind == QT_SWAP) {
        HostOp op;
        op.kind = OP_SWAP;
        op.q0 = std::min(g.target[0], g.target[1]);
        op.q1 = std::max(g.target[0], g.target[1]);
        out->push_back(op);
        return true;
    }
    M2 U;
    if (!base_matrix(g, &U)) {
        *err = "no matrix for kind";
        return false;
    }
    uint64_t cmask = 0;
    for (int k = 0; k < g.ncontrol; ++k) cmask |= uint64_t(1) << g.control[k];
    out->push_back(classify(U, g.target[0], cmask, 1));
    return true;
}

bool Pass::same_as(const Pass& o) const {
    if (lt != o.lt || nh != o.nh || ops.size() != o.ops.size() || blocks.size() != o.blocks.size()) return false;
    for (size_t b = 0; b < blocks.size(); ++b) {
        if (std::memcmp(blocks[b].q, o.blocks[b].q, sizeof blocks[b].q) != 0 || blocks[b].u != o.blocks[b].u)
            return false;
    }
    for (int k = 0; k < nh; ++k)
        if (h[k] != o.h[k]) return false;
    for (size_t i = 0; i < ops.size(); ++i) {
        const HostOp &a = ops[i], &b = o.ops[i];
        if (a.kind != b.kind || a.q0 != b.q0 || a.q1 != b.q1 || a.cmask != b.cmask || a.ngates != b.ngates)
            return false;
        if (std::memcmp(a.m, b.m, sizeof a.m) != 0) return false;
    }
    return true;
}

// Greedy tile fusion over a segment.  Gates come in canonical order (levels
// in order, each level by ascending lowest qubit).  A pass collects, in order,
// every gate that (a) does not depend on a gate left out of the pass (shares
// no qubit with one), and (b) keeps the set of tile qubits at or above lt
// within nh_max.  Diagonal ops and controls need no tile qubit: on a qubit
// outside the tile they are uniform over the tile.  Consecutive one-qubit ops
// on the same qubit are then multiplied into one 2x2 (FP64, on the host).
SegPlan plan_segment(const std::vector<const qt_gate*>& gates, const PlanParams& pp) {
    SegPlan sp;
    struct Item {
        std::vector<HostOp> ops;
        uint64_t qubits;
        uint64_t need;  // qubits >= lt that must be tile qubits
    };
    std::vector<Item> items;
    items.reserve(gates.size());
    for (const qt_gate* g : gates) {
        Item it;
        std::string err;
        lower_gate(*g, pp.n, &it.ops, &err);
        it.qubits = gate_qubit_mask(*g);
        it.need = 0;
        for (const HostOp& op : it.ops) {
            if (is_diagonal(op)) continue;
            if (op.q0 >= pp.lt) it.need |= uint64_t(1) << op.q0;
            if (op.q1 >= pp.lt) it.need |= uint64_t(1) << op.q1;
        }
        items.push_back(std::move(it));
    }
    std::vector<char> done(items.size(), 0);
    size_t ndone = 0;
    const uint32_t nparts_bits = pp.n - pp.p;
    while (ndone < items.size()) {
        Pass ps;
        uint64_t H = 0, blocked = 0;
        std::vector<HostOp> ops;
        for (size_t i = 0; i < items.size(); ++i) {
            if (done[i]) continue;
            const Item& it = items[i];
            if (it.qubits & blocked) {
                blocked |= it.qubits;
                continue;
            }
            uint64_t nH = H | it.need;
            bool fits = popcount64(nH) <= pp.nh_max;
            // The first unscheduled gate always starts a pass, even when its
            // targets exceed nh_max (a SWAP on two high qubits with
            // nh_max = 1): every sweep makes progress.
            if (ops.empty() && ps.ngates == 0) fits = true;
            if (!pp.fusion && !ops.empty()) fits = false;
            if (!fits) {
                blocked |= it.qubits;
                continue;
            }
            H = nH;
            for (const HostOp& op : it.ops) ops.push_back(op);
            ps.ngates += 1;
            done[i] = 1;
            ++ndone;
        }
        // Merge consecutive one-qubit ops on the same qubit.
        std::vector<HostOp> merged;
        std::vector<int> last(pp.n, -1);  // index into merged of the last op touching q
        for (const HostOp& op : ops) {
            uint64_t qs = op_qubits(op);
            if (pp.merge && single_qubit(op) && last[op.q0] >= 0 && single_qubit(merged[last[op.q0]]) &&
                merged[last[op.q0]].q0 == op.q0) {
                HostOp& prev = merged[last[op.q0]];
                M2 a, b;
                op_matrix(prev, &a);
                op_matrix(op, &b);
                HostOp m = classify(mul(b, a), op.q0, 0, prev.ngates + op.ngates);
                if (op_cost(m) <= op_cost(prev) + op_cost(op)) {  // merge only when it saves work
                    prev = m;
                    continue;
                }
            }
            merged.push_back(op);
            for (int q = 0; q < pp.n; ++q)
                if ((qs >> q) & 1) last[q] = int(merged.size()) - 1;
        }
        // Drop exact identities left by merging.
        for (const HostOp& op : merged) {
            bool ident = false;
            if (op.kind == OP_PHASE && op.m[0] == 1.0 && op.m[1] == 0.0) ident = true;
            if (op.kind == OP_DIAG && op.m[0] == 1.0 && op.m[1] == 0.0 && op.m[2] == 1.0 && op.m[3] == 0.0)
                ident = true;
            if (!ident) ps.ops.push_back(op);
        }
        ps.lt = pp.lt;
        // Pad the tile to its full size with qubits inside the partition
        // (they add no coupling between partitions): larger tiles amortise
        // the per-op work over more amplitudes per thread and keep every
        // pass on the register kernel.
        for (int q = pp.lt; q < std::min(pp.p, pp.n) && popcount64(H) < pp.nh_max; ++q)
            H |= uint64_t(1) << q;
        ps.nh = 0;
        for (int q = pp.lt; q < pp.n; ++q)
            if ((H >> q) & 1) ps.h[ps.nh++] = q;
        ps.M = 0;
        for (int k = 0; k < ps.nh; ++k)
            if (ps.h[k] >= pp.p) ps.M |= uint32_t(1) << (ps.h[k] - pp.p);
        // Support: partitions where some op can act -- its partition-level
        // conditions (controls and phase qubits at or above p) all hold.
        ps.supp_all = false;
        for (const HostOp& op : ps.ops) {
            uint32_t pm = nparts_bits ? uint32_t(op.cmask >> pp.p) : 0;
            if (pm == 0) ps.supp_all = true;
            ps.supp_masks.push_back(pm);
        }
        if (ps.ops.empty()) ps.supp_all = false;  // a pass reduced to nothing touches nothing
        if (pp.tc_blocks && ps.lt == 7 && ps.nh == 5) fuse_blocks(&ps, pp);
        if (ps.ngates > 0) sp.passes.push_back(std::move(ps));
    }
    return sp;
}

// ------------------------------------------------------ tensor-core blocks --
namespace {

// Register-kernel cost of an op in units of one dense one-qubit op
// (complex64, measured per-op costs: dense 2x2 0.13 SM-cycles per amplitude,
// real 2x2 ~0.09, controlled phases and exchanges ~0.05, relabels ~0).
double reg_cost(const HostOp& op) {
    switch (op.kind) {
        case OP_DENSE: return 1.0;
        case OP_REAL: case OP_IREAL: case OP_ANTI: case OP_DIAG: return 0.7;
        case OP_PHASE: return 0.4;
        case OP_X: case OP_SWAP: return op.cmask ? 0.6 : 0.05;
        default: return 1.0;
    }
}

// Apply op (acting on qubits inside the block) to the columns of the 32x32
// matrix u (row-major complex): u := M_op u.  pos[q] = block bit of qubit q.
void block_apply(std::vector<cd>& u, const HostOp& op, const int* pos) {
    uint32_t cm = 0;
    for (int q = 0; q < 64; ++q)
        if ((op.cmask >> q) & 1) cm |= 1u << pos[q];
    auto ok = [&](uint32_t r) { return (r & cm) == cm; };
    for (int col = 0; col < 32; ++col) {
        auto U = [&](uint32_t r) -> cd& { return u[size_t(r) * 32 + col]; };
        switch (op.kind) {
            case OP_DENSE: case OP_REAL: case OP_IREAL: case OP_X: case OP_ANTI: {
                const uint32_t t = 1u << pos[op.q0];
                M2 m;
                op_matrix(op, &m);
                for (uint32_t r = 0; r < 32; ++r) {
                    if ((r & t) || !ok(r)) continue;
                    const cd a = U(r), b = U(r | t);
                    U(r) = m.a[0] * a + m.a[1] * b;
                    U(r | t) = m.a[2] * a + m.a[3] * b;
                }
                break;
            }
            case OP_SWAP: {
                const uint32_t t0 = 1u << pos[op.q0], t1 = 1u << pos[op.q1];
                for (uint32_t r = 0; r < 32; ++r)
                    if ((r & t0) && !(r & t1) && ok(r)) std::swap(U(r), U(r ^ t0 ^ t1));
                break;
            }
            case OP_DIAG: {
                const uint32_t t = 1u << pos[op.q0];
                for (uint32_t r = 0; r < 32; ++r)
                    if (ok(r)) U(r) *= (r & t) ? get(op.m, 1) : get(op.m, 0);
                break;
            }
            case OP_PHASE:
                for (uint32_t r = 0; r < 32; ++r)
                    if (ok(r)) U(r) *= get(op.m, 0);
                break;
            default: break;
        }
    }
}

}  // namespace

void fuse_blocks(Pass* ps, const PlanParams& pp) {
    uint64_t tile = (uint64_t(1) << ps->lt) - 1;
    for (int k = 0; k < ps->nh; ++k) tile |= uint64_t(1) << ps->h[k];
    std::vector<HostOp> out;
    std::vector<HostOp> cur;
    uint64_t cq = 0;
    double ccost = 0.0;
    auto flush = [&]() {
        if (cur.empty()) return;
        if (ccost < pp.tc_threshold) {
            for (const HostOp& o : cur) out.push_back(o);
        } else {
            // pad to five qubits with the highest other tile qubits (the rows
            // keep the low ones, which become lane bits: coalesced stores)
            Block b;
            int nq = 0;
            for (int q = 0; q < 64; ++q)
                if ((cq >> q) & 1) b.q[nq++] = q;
            for (int q = 63; q >= 0 && nq < 5; --q)
                if (((tile >> q) & 1) && !((cq >> q) & 1)) {
                    cq |= uint64_t(1) << q;
                    b.q[nq++] = q;
                }
            std::sort(b.q, b.q + 5);
            int pos[64];
            for (int i = 0; i < 5; ++i) pos[b.q[i]] = i;
            std::vector<cd> u(32 * 32, cd(0.0, 0.0));
            for (int i = 0; i < 32; ++i) u[size_t(i) * 32 + i] = 1.0;
            int ng = 0;
            for (const HostOp& o : cur) {
                block_apply(u, o, pos);
                ng += o.ngates;
            }
            b.u.resize(2 * 32 * 32);
            for (size_t i = 0; i < u.size(); ++i) {
                b.u[2 * i] = u[i].real();
                b.u[2 * i + 1] = u[i].imag();
            }
            HostOp bo;
            bo.kind = OP_BLOCK;
            bo.q0 = int32_t(ps->blocks.size());
            bo.cmask = 0;
            bo.ngates = ng;
            ps->blocks.push_back(std::move(b));
            out.push_back(bo);
        }
        cur.clear();
        cq = 0;
        ccost = 0.0;
    };
    for (const HostOp& o : ps->ops) {
        const uint64_t q = op_qubits(o);
        const bool eligible = (q & ~tile) == 0 && o.kind != OP_BLOCK;
        if (eligible && popcount64(cq | q) <= 5) {
            cur.push_back(o);
            cq |= q;
            ccost += reg_cost(o);
            continue;
        }
        if (!eligible && (q & cq) == 0) {  // commutes with every op of the block: runs before it
            out.push_back(o);
            continue;
        }
        flush();
        if (eligible) {
            cur.push_back(o);
            cq = q;
            ccost = reg_cost(o);
        } else {
            out.push_back(o);
        }
    }
    flush();
    ps->ops.swap(out);
}

void block_operand(const Block& b, float* out) {
    auto tf32 = [](float f) {  // round to the nearest tf32 (10 fraction bits), ties away from zero
        uint32_t u;
        std::memcpy(&u, &f, 4);
        u = (u + 0x1000u) & ~0x1FFFu;
        float r;
        std::memcpy(&r, &u, 4);
        return r;
    };
    std::memset(out, 0, kBlockBytes);
    float* hi = out;
    float* lo = out + kBlockBytes / 8;
    for (int n = 0; n < 64; ++n) {
        for (int k = 0; k < 64; ++k) {
            // real embedding: out(2j'+c') = sum_k W[n][k] in(2j+c)
            const int jo = n >> 1, ji = k >> 1;
            const double ur = b.u[2 * (size_t(jo) * 32 + ji)], ui = b.u[2 * (size_t(jo) * 32 + ji) + 1];
            const int co = n & 1, ci = k & 1;
            const double w = co == 0 ? (ci == 0 ? ur : -ui) : (ci == 0 ? ui : ur);
            const float h = tf32(float(w));
            const float l = tf32(float(w - double(h)));
            // K-major, 128-byte swizzle: two K atoms of 32 elements, rows of 128 B,
            // 16-byte chunk c of row n stored at chunk c ^ (n % 8)
            const size_t byte = size_t(k / 32) * 8192 + size_t(n / 8) * 1024 + size_t(n % 8) * 128 +
                                size_t((((k % 32) / 4) ^ (n % 8)) * 16) + size_t(k % 4) * 4;
            hi[byte / 4] = h;
            lo[byte / 4] = l;
        }
    }
}

// ------------------------------------------------------------ bitsets ---

bool Bitset::all() const {
    for (uint32_t i = 0; i + 1 < w.size(); ++i)
        if (w[i] != ~uint64_t(0)) return false;
    if (w.empty()) return true;
    uint64_t lastmask = (nbits & 63) ? (uint64_t(1) << (nbits & 63)) - 1 : ~uint64_t(0);
    return w.back() == lastmask;
}

uint64_t Bitset::count() const {
    uint64_t c = 0;
    for (auto x : w) c += __builtin_popcountll(x);
    return c;
}

bool Bitset::or_with(const Bitset& o) {
    bool ch = false;
    for (size_t i = 0; i < w.size(); ++i) {
        uint64_t nw = w[i] | o.w[i];
        ch = ch || nw != w[i];
        w[i] = nw;
    }
    return ch;
}

Bitset pass_support(const Pass& ps, uint32_t nparts) {
    Bitset s;
    s.resize(nparts);
    if (ps.supp_all) {
        s.fill();
        return s;
    }
    for (uint32_t pm : ps.supp_masks)
        for (uint32_t q = 0; q < nparts; ++q)
            if ((q & pm) == pm) s.set(q);
    return s;
}

namespace {
// Mark every member of each coupling group that meets T.
bool mark_groups(Bitset* D, const Bitset& T, uint32_t M) {
    bool changed = false;
    for (size_t wi = 0; wi < T.w.size(); ++wi) {
        uint64_t word = T.w[wi];
        while (word) {
            int b = __builtin_ctzll(word);
            word &= word - 1;
            uint32_t q = uint32_t(wi * 64 + b);
            uint32_t g = q & ~M;
            uint32_t m = 0;
            do {
                uint32_t r = g | m;
                if (!D->get(r)) {
                    D->set(r);
                    changed = true;
                }
                m = (m - M) & M;
            } while (m != 0);
        }
    }
    return changed;
}
}  // namespace

void close_forward(Bitset* D, const Pass& ps, const Bitset& supp) {
    if (ps.M == 0 || D->all()) return;
    Bitset T = *D;
    for (size_t i = 0; i < T.w.size(); ++i) T.w[i] &= supp.w[i];
    mark_groups(D, T, ps.M);
}

void close_all(Bitset* W, const std::vector<Pass>& passes, const std::vector<Bitset>& supps) {
    bool changed = true;
    while (changed && !W->all()) {
        changed = false;
        for (size_t i = 0; i < passes.size(); ++i) {
            if (passes[i].M == 0) continue;
            Bitset T = *W;
            for (size_t k = 0; k < T.w.size(); ++k) T.w[k] &= supps[i].w[k];
            changed = mark_groups(W, T, passes[i].M) || changed;
        }
    }
}

// ------------------------------------------------ merged phase groups --
namespace {

bool is_phase_code(uint8_t c) { return c >= RC_PH_NEG && c <= RC_PH_GEN; }
bool is_diag_code(uint8_t c) { return is_phase_code(c) || (c >= RC_DIAG_G && c <= RC_DIAG_R); }

// A resolved phase op that can be a term of a group: every amplitude of the
// thread, or those with one (unflipped) register bit set.
bool groupable(const DevOp& o) { return is_phase_code(o.rh.code) && o.rh.mcls <= 1 && o.rh.ren == 0; }

// Estimated per-thread work in units of one complex multiply: an op's fixed
// decode cost, then its multiplies (a +-1 / +-i phase is a sign change and a
// move, not a multiply).
struct PhaseCost {
    double op, move;
    explicit PhaseCost(int coef_bytes)
        : op(coef_bytes == 8 ? 4.0 : 0.4), move(coef_bytes == 8 ? 0.5 : 0.1) {}
    double single(const DevOp& o, int R) const {
        const double regs = o.rh.mcls == 0 ? R : o.rh.mcls == 1 ? R / 2.0 : R / 4.0;
        return op + regs * (o.rh.code == RC_PH_GEN ? 1.0 : move);
    }
    double group(int nterms, int nsteps, double regs) const { return op * (1 + 0.5 * nsteps) + 1.25 * nterms + regs; }
};

// Emit the merged group of the terms in `m` (all groupable): one step for the
// terms on every register of the thread, one per register bit.
void emit_group(std::vector<DevOp>* out, const std::vector<const DevOp*>& m, int coef_bytes, int nreg) {
    std::vector<PhTerm> terms;
    for (int cls = -1; cls < nreg; ++cls) {
        const size_t first = terms.size();
        for (const DevOp* o : m) {
            const int oc = o->rh.mcls == 0 ? -1 : o->rh.a;
            if (oc != cls) continue;
            PhTerm t;
            std::memset(&t, 0, sizeof t);
            std::memcpy(&t.f, &o->m, size_t(coef_bytes));
            t.cm_glob = o->cm_glob;
            t.cm_thr = uint16_t(o->rh.cm_thr);
            t.cv_thr = uint16_t(o->rh.cv_thr);
            t.mcls = cls < 0 ? 0 : 1;
            t.k = uint8_t(cls < 0 ? 0 : cls);
            terms.push_back(t);
        }
        if (terms.size() > first) terms.back().last = 1;
    }
    DevOp h;
    std::memset(&h, 0, sizeof h);
    h.kind = OP_PHASE;
    h.b0 = -1;
    h.b1 = int32_t(terms.size());
    h.rh.code = RC_PH_GROUP;
    // bit i: term i is the last of its step (the kernel walks the steps by it)
    uint64_t ends = 0;
    for (size_t i = 0; i < terms.size(); ++i)
        if (terms[i].last) ends |= uint64_t(1) << i;
    static_assert(sizeof(h.perm) == sizeof(ends), "step-end mask fits the header's perm field");
    std::memcpy(h.perm, &ends, sizeof ends);
    out->push_back(h);
    for (size_t i = 0; i < terms.size(); i += kTermsPerSlot) {
        DevOp slot;
        std::memset(&slot, 0, sizeof slot);
        std::memcpy(&slot, terms.data() + i, sizeof(PhTerm) * std::min<size_t>(kTermsPerSlot, terms.size() - i));
        out->push_back(slot);
    }
}

// Replace runs of consecutive diagonal ops (which commute) by a merged group
// of their groupable phases, the rest of the run after it, when the estimate
// says the group costs less; then pad with NOP ops so that no group's header
// and term slots straddle two staging chunks.
bool merge_phase_groups(std::vector<DevOp>* ops_io, int coef_bytes, int nreg) {
    std::vector<DevOp>& ops = *ops_io;
    const int R = 1 << nreg;
    const PhaseCost cost(coef_bytes);
    constexpr int kMaxTerms = 15 * kTermsPerSlot;  // 60: the kernel tracks a group's terms in one 64-bit mask
    std::vector<DevOp> out;
    bool any = false;
    size_t i = 0;
    while (i < ops.size()) {
        if (!is_diag_code(ops[i].rh.code)) {
            out.push_back(ops[i++]);
            continue;
        }
        size_t j = i;
        while (j < ops.size() && is_diag_code(ops[j].rh.code)) ++j;
        std::vector<const DevOp*> m, rest;
        for (size_t k = i; k < j; ++k) (groupable(ops[k]) ? m : rest).push_back(&ops[k]);
        for (size_t g0 = 0; g0 < m.size(); g0 += kMaxTerms) {
            std::vector<const DevOp*> part(m.begin() + long(g0), m.begin() + long(std::min(m.size(), g0 + kMaxTerms)));
            double now = 0.0, regs = 0.0;
            uint32_t steps = 0;
            for (const DevOp* o : part) {
                now += cost.single(*o, R);
                steps |= o->rh.mcls == 0 ? 1u : 2u << o->rh.a;
            }
            for (int b = 0; b <= nreg; ++b)
                if ((steps >> b) & 1u) regs += b == 0 ? R : R / 2.0;
            if (part.size() >= 2 && cost.group(int(part.size()), __builtin_popcount(steps), regs) < 0.9 * now) {
                emit_group(&out, part, coef_bytes, nreg);
                any = true;
            } else
                for (const DevOp* o : part) out.push_back(*o);
        }
        for (const DevOp* o : rest) out.push_back(*o);
        i = j;
    }
    // pad: a group's header and its slots stay inside one chunk
    std::vector<DevOp> padded;
    padded.reserve(out.size());
    for (size_t k = 0; k < out.size();) {
        size_t len = 1;
        if (out[k].rh.code == RC_PH_GROUP) len += size_t((out[k].b1 + kTermsPerSlot - 1) / kTermsPerSlot);
        const size_t pos = padded.size() % kOpChunk;
        if (pos + len > size_t(kOpChunk)) {
            DevOp nop;
            std::memset(&nop, 0, sizeof nop);
            nop.kind = OP_PHASE;
            nop.b0 = -1;
            nop.rh.code = RC_NOP;
            while (padded.size() % kOpChunk != 0) padded.push_back(nop);
        }
        for (size_t q = 0; q < len; ++q) padded.push_back(out[k + q]);
        k += len;
    }
    ops.swap(padded);
    return any;
}

}  // namespace

// ------------------------------------------------ register-kernel layout --
// The register kernel holds each tile bit on a lane-id bit, a register-index
// bit or a warp-id bit.  The ops are walked in order, tracking that layout
// (TileLayout, with the flip of pending X gates):
//  - an uncontrolled X only toggles the flip, an uncontrolled SWAP only
//    exchanges the two tile bits' places: neither becomes a kernel op;
//  - before the first op with a target on a warp bit, an OP_PERM moves (via
//    shared memory) to a layout whose register bits hold that op's targets
//    and as many of the following ops' targets as fit (then bits of the old
//    layout, then the highest tile bits), lane bit i holding tile bit i, and
//    applies the flip;
//  - every other op is resolved against the current layout: targets and
//    conditions become physical bits, a flipped target exchanges the op's
//    matrix entries (X U X), a flipped condition is marked in the value mask.
void set_register_offsets(DevPass* dp) {
    // tile bit b < lt is amplitude-index bit b; tile bit lt + k is qubit h[k]
    auto off = [dp](int b) -> uint64_t { return uint64_t(1) << (b < dp->lt ? b : dp->h[b - dp->lt]); };
    for (int k = 0; k < kMaxRegBits; ++k) {
        dp->rin[k] = k < dp->nreg ? off(dp->layout[k]) : 0;
        dp->rout[k] = k < dp->nreg ? off(dp->fin.reg[k]) : 0;
    }
}

void plan_register_layout(DevPass* dp, std::vector<DevOp>* ops_io, int coef_bytes, bool reorder, bool phase_groups,
                          bool dense_regk) {
    const int tb = dp->lt + dp->nh;
    dp->reg_kernel = 0;
    dp->groups = 0;
    if (tb < 7) return;
    const int nreg = std::min(5, std::max(2, tb - 8));
    const int nwarp = tb - 5 - nreg;
    dp->reg_kernel = 1;
    dp->nreg = nreg;
    dp->nwarp = nwarp;
    std::vector<DevOp>& ops = *ops_io;
    const uint32_t upper = ((1u << tb) - 1u) & ~31u;
    auto relabel = [](const DevOp& o) {
        return (o.kind == OP_X || o.kind == OP_SWAP) && o.cm_glob == 0 && o.cm_tile == 0;
    };
    auto targets = [](const DevOp& o) -> uint32_t {
        switch (o.kind) {
            case OP_DENSE: case OP_REAL: case OP_IREAL: case OP_X: case OP_ANTI: return 1u << o.b0;
            case OP_SWAP: return (1u << o.b0) | (1u << o.b1);
            default: return 0u;  // a tensor-core block reads any layout
        }
    };
    auto block_bits = [](const DevOp& o) -> uint32_t {
        const BlockStage& bs = *reinterpret_cast<const BlockStage*>(&o.m);
        uint32_t m = 0;
        for (int i = 0; i < 5; ++i) m |= 1u << bs.s[i];
        return m;
    };
    dp->mma = 0;
    auto pc = [](uint32_t x) { return __builtin_popcount(x); };
    std::vector<char> done(ops.size(), 0);
    // register set of a new layout for op i and the ops not yet placed after
    // it: their targets above the lanes.  A pass whose ops all merged into
    // identities has none: its layout is just the highest tile bits.
    auto choose = [&](size_t i, uint32_t keep) -> uint32_t {
        uint32_t s = i < ops.size() ? targets(ops[i]) & upper : 0u;
        for (size_t j = 0; j < ops.size(); ++j) {
            if (j == i || done[j] || relabel(ops[j])) continue;
            const uint32_t t = s | (targets(ops[j]) & upper);
            if (pc(t) > nreg) break;
            s = t;
        }
        for (int b = tb - 1; b >= 5 && pc(s) < nreg; --b)
            if ((keep >> b) & 1u) s |= 1u << b;
        for (int b = tb - 1; b >= 5 && pc(s) < nreg; --b)
            if ((upper >> b) & 1u) s |= 1u << b;
        return s;
    };
    // where[t]: 0..4 lane bit, 8 + k register bit k, 16 + w warp bit w
    TileLayout L;
    int where[32];
    auto set_layout = [&](uint32_t regset) {
        std::memset(&L, 0, sizeof L);
        int k = 0, w = 0;
        for (int b = 0; b < 5; ++b) L.lane[b] = int8_t(b);
        for (int b = 5; b < tb; ++b) {
            if ((regset >> b) & 1u) L.reg[k++] = int8_t(b);
            else L.warp[w++] = int8_t(b);
        }
        for (int b = 0; b < 5; ++b) where[b] = b;
        for (int j = 0; j < nreg; ++j) where[L.reg[j]] = 8 + j;
        for (int j = 0; j < nwarp; ++j) where[L.warp[j]] = 16 + j;
    };
    auto placed = [&](uint32_t tm) {
        for (int t = 0; t < tb; ++t)
            if (((tm >> t) & 1u) && where[t] >= 16) return false;
        return true;
    };
    uint32_t cur = choose(0, 0);
    set_layout(cur);
    for (int k = 0; k < nreg; ++k) dp->layout[k] = L.reg[k];
    for (int w = 0; w < nwarp; ++w) dp->layout[nreg + w] = L.warp[w];
    auto emit_perm = [&](std::vector<DevOp>& out, uint32_t regset) {
        DevOp pm;
        std::memset(&pm, 0, sizeof pm);
        pm.kind = OP_PERM;
        pm.rh.code = RC_PERM;
        pm.nreg = int8_t(nreg);
        pm.nwarp = int8_t(nwarp);
        static_assert(sizeof(TileLayout) <= sizeof(pm.m), "old layout fits the matrix field");
        std::memcpy(&pm.m, &L, sizeof L);
        set_layout(regset);
        for (int k = 0; k < nreg; ++k) pm.perm[k] = L.reg[k];
        for (int w = 0; w < nwarp; ++w) pm.perm[nreg + w] = L.warp[w];
        out.push_back(pm);
    };
    auto swap_entries = [&](DevOp& o, int i, int j) {
        unsigned char* m = reinterpret_cast<unsigned char*>(&o.m);
        unsigned char t[16];
        std::memcpy(t, m + i * coef_bytes, size_t(coef_bytes));
        std::memcpy(m + i * coef_bytes, m + j * coef_bytes, size_t(coef_bytes));
        std::memcpy(m + j * coef_bytes, t, size_t(coef_bytes));
    };
    // Ops that commute (no common tile bit, or both diagonal) may run in any
    // order.  The ops are taken in list order, except that when the next op
    // would need a layout change, a later ready op whose targets are already
    // placed goes first (option `reorder`, on by default).
    const size_t n = ops.size();
    std::vector<uint32_t> qm(n);
    std::vector<char> dg(n);
    for (size_t i = 0; i < n; ++i) {
        // every tile bit the op reads or changes (a DIAG outside the tile is a
        // factor per tile and touches none)
        qm[i] = targets(ops[i]) | ops[i].cm_tile;
        if (ops[i].kind == OP_DIAG && ops[i].b0 >= 0) qm[i] |= 1u << ops[i].b0;
        if (ops[i].kind == OP_BLOCK) qm[i] = block_bits(ops[i]);
        dg[i] = ops[i].kind == OP_DIAG || ops[i].kind == OP_PHASE;
    }
    auto commute = [&](size_t i, size_t j) { return (qm[i] & qm[j]) == 0 || (dg[i] && dg[j]); };
    std::vector<int> npred(n, 0);
    for (size_t j = 0; j < n; ++j)
        for (size_t i = 0; i < j; ++i)
            if (!commute(i, j)) ++npred[j];
    auto ready_without_perm = [&](const DevOp& c) {
        if (relabel(c)) return true;
        const bool mixed = c.kind == OP_SWAP && (((L.flip >> c.b0) ^ (L.flip >> c.b1)) & 1u);
        return placed(targets(c)) && !mixed;
    };
    std::vector<DevOp> out;
    out.reserve(ops.size() + 4);
    for (size_t step = 0; step < n; ++step) {
        size_t i = n, first = n;
        for (size_t k = 0; k < n; ++k) {
            if (done[k] || npred[k] != 0) continue;
            if (first == n) first = k;
            if (!reorder || ready_without_perm(ops[k])) {
                i = k;
                break;
            }
        }
        if (i == n) i = first;
        done[i] = 1;
        for (size_t j = i + 1; j < n; ++j)
            if (!done[j] && !commute(i, j)) --npred[j];
        DevOp o = ops[i];
        if (o.kind == OP_BLOCK) {
            // tensor-core block: record, for each physical bit and the flip,
            // the operand-A byte offset its tile bit contributes (row or block
            // index), then take the fixed post-MMA layout
            BlockStage& bs = *reinterpret_cast<BlockStage*>(&o.m);
            auto contrib = [&](int t) -> uint16_t {
                for (int i = 0; i < 5; ++i)
                    if (bs.s[i] == t) return uint16_t(block_a_offset(0u, 1u << i));
                for (int i = 0; i < 7; ++i)
                    if (bs.rows[i] == t) return uint16_t(block_a_offset(1u << i, 0u));
                return 0;
            };
            for (int b = 0; b < 5; ++b) bs.a_lane[b] = contrib(L.lane[b]);
            for (int k = 0; k < 4; ++k) bs.a_reg[k] = k < nreg ? contrib(L.reg[k]) : 0;
            for (int w = 0; w < 3; ++w) bs.a_warp[w] = w < nwarp ? contrib(L.warp[w]) : 0;
            bs.a_flip = 0;
            for (int t = 0; t < tb; ++t)
                if ((L.flip >> t) & 1u) bs.a_flip ^= contrib(t);
            std::memset(&L, 0, sizeof L);
            for (int b = 0; b < 5; ++b) L.lane[b] = bs.rows[b];
            for (int k = 0; k < 4; ++k) L.reg[k] = bs.s[k];
            L.warp[0] = bs.rows[5];
            L.warp[1] = bs.rows[6];
            L.warp[2] = bs.s[4];
            for (int b = 0; b < 5; ++b) where[L.lane[b]] = b;
            for (int k = 0; k < 4; ++k) where[L.reg[k]] = 8 + k;
            for (int w = 0; w < 3; ++w) where[L.warp[w]] = 16 + w;
            cur = 0;
            for (int k = 0; k < 4; ++k) cur |= 1u << L.reg[k];
            std::memset(&o.rh, 0, sizeof o.rh);
            o.rh.code = RC_MMA;
            dp->mma = 1;
            out.push_back(o);
            continue;
        }
        if (relabel(o)) {
            if (o.kind == OP_X) {
                L.flip ^= 1u << o.b0;
            } else {
                const int t1 = o.b0, t2 = o.b1, p1 = where[t1], p2 = where[t2];
                auto slot = [&](int p) -> int8_t& { return p < 8 ? L.lane[p] : p < 16 ? L.reg[p - 8] : L.warp[p - 16]; };
                slot(p1) = int8_t(t2);
                slot(p2) = int8_t(t1);
                where[t1] = p2;
                where[t2] = p1;
                const uint32_t f1 = (L.flip >> t1) & 1u, f2 = (L.flip >> t2) & 1u;
                L.flip = (L.flip & ~((1u << t1) | (1u << t2))) | (f1 << t2) | (f2 << t1);
            }
            continue;
        }
        const uint32_t tg = targets(o);
        // a conditioned SWAP whose two bits are flipped differently exchanges
        // another pair of patterns: apply the flip with a layout change first
        const bool swap_mixed = o.kind == OP_SWAP && (((L.flip >> o.b0) ^ (L.flip >> o.b1)) & 1u);
        if (!placed(tg) || swap_mixed) {
            cur = choose(i, cur);
            emit_perm(out, cur);
        }
        const uint32_t F = L.flip;
        // conditions on physical bits, flipped ones marked in the value masks
        uint32_t thr = 0, cvt = 0;
        uint16_t reg = 0;
        uint8_t cvr = 0;
        for (int b = 0; b < tb; ++b) {
            if (!((o.cm_tile >> b) & 1u)) continue;
            const int p = where[b];
            const uint32_t f = (F >> b) & 1u;
            if (p >= 8 && p < 16) {
                reg |= uint16_t(1u << (p - 8));
                cvr |= uint8_t(f << (p - 8));
            } else {
                const int tbit = p < 8 ? p : 5 + (p - 16);
                thr |= 1u << tbit;
                cvt |= f << tbit;
            }
        }
        RegHdr h;
        std::memset(&h, 0, sizeof h);
        h.code = RC_NOP;
        const bool pair = o.kind == OP_DENSE || o.kind == OP_REAL || o.kind == OP_IREAL || o.kind == OP_X ||
                          o.kind == OP_ANTI;
        if (pair) {
            if ((F >> o.b0) & 1u) {  // X U X: the stored pair is exchanged
                if (o.kind == OP_DENSE || o.kind == OP_REAL || o.kind == OP_IREAL) {
                    swap_entries(o, 0, 3);
                    swap_entries(o, 1, 2);
                } else if (o.kind == OP_ANTI) {
                    swap_entries(o, 0, 1);
                }
            }
            const int cr = o.kind == OP_DENSE ? RC_DENSE_R : o.kind == OP_REAL ? RC_REAL_R
                         : o.kind == OP_IREAL ? RC_IREAL_R : o.kind == OP_X ? RC_X_R : RC_ANTI_R;
            const int p = where[o.b0];
            if (p < 8) {
                h.code = uint8_t(cr + 1);  // the _L variant
                h.a = int8_t(p);
            } else {
                const int k = p - 8;
                h.code = uint8_t(cr);
                if (k > 0 && dense_regk && o.kind == OP_DENSE) {
                    h.b = int8_t(k);  // pairs across register bit k, layout unchanged
                } else if (k > 0) {
                    // the kernel exchanges register bits 0 and k first
                    h.ren = int8_t(k);
                    auto x0k = [k](uint32_t v) -> uint32_t {
                        const uint32_t b0 = v & 1u, bk = (v >> k) & 1u;
                        return (v & ~(1u | (1u << k))) | (b0 << k) | bk;
                    };
                    reg = uint16_t(x0k(reg));
                    cvr = uint8_t(x0k(cvr));
                    const int t0 = L.reg[0], tk = L.reg[k];
                    L.reg[0] = int8_t(tk);
                    L.reg[k] = int8_t(t0);
                    where[tk] = 8;
                    where[t0] = 8 + k;
                }
            }
        } else if (o.kind == OP_SWAP) {
            const int p0 = where[o.b0], p1 = where[o.b1];
            if (p0 < 8 && p1 < 8) {
                h.code = RC_SWAP_LL;
                h.a = int8_t(p0);
                h.b = int8_t(p1);
            } else if (p0 < 8 || p1 < 8) {
                h.code = RC_SWAP_LR;
                h.a = int8_t(p0 < 8 ? p0 : p1);
                h.b = int8_t((p0 < 8 ? p1 : p0) - 8);
            } else {
                h.code = RC_SWAP_RR;
                h.a = int8_t(std::min(p0, p1) - 8);
                h.b = int8_t(std::max(p0, p1) - 8);
            }
        } else if (o.kind == OP_DIAG) {
            if (o.b0 < 0) {
                h.code = RC_DIAG_G;
                h.a = int8_t(o.gq);
            } else {
                if ((F >> o.b0) & 1u) swap_entries(o, 0, 1);
                const int p = where[o.b0];
                if (p >= 8 && p < 16) {
                    h.code = RC_DIAG_R;
                    h.a = int8_t(p - 8);
                } else {
                    h.code = RC_DIAG_T;
                    h.a = int8_t(p < 8 ? p : 5 + (p - 16));
                }
            }
        } else if (o.kind == OP_PHASE) {
            h.code = o.sub == PH_NEG ? RC_PH_NEG : o.sub == PH_POS_I ? RC_PH_POS_I
                   : o.sub == PH_NEG_I ? RC_PH_NEG_I : RC_PH_GEN;
            h.mcls = reg == 0 ? 0 : ((reg & (reg - 1)) == 0 && cvr == 0) ? 1 : 2;
            if (h.mcls == 1) h.a = int8_t(__builtin_ctz(reg));
        }
        h.cm_reg = reg;
        h.cv_reg = cvr;
        h.cm_thr = thr;
        h.cv_thr = cvt;
        o.rh = h;
        out.push_back(o);
    }
    dp->fin = L;
    ops.swap(out);
    if (phase_groups) dp->groups = merge_phase_groups(&ops, coef_bytes, nreg) ? 1 : 0;
}

}  // namespace qt
