// Host check of the register-kernel layout planner (plan_register_layout).
//
// For random circuits, every fused pass is planned twice over the same
// tile-local ops:
//   reference  the encoded ops applied in list order to a logical tile
//              (targets and conditions as tile-index bits, global
//              conditions read from a random tile base);
//   planned    the planner's output -- dispatch codes on physical lane,
//              register and warp bits, register renames, layout changes,
//              relabels with their flip mask -- executed with the register
//              kernel's semantics on a physical tile, then stored through the
//              final layout.
// Both use exact binary64 complex arithmetic on random tile contents; the
// results must agree to rounding.  A second part plans complex64-shaped
// passes (tiles of 12 qubits) with tensor-core blocks and checks the fused
// blocks (their FP64 matrices, the ops moved ahead of them, the staging
// masks and the layout after each block) the same way.  Each pass's register
// offsets (the kernel's amplitude addressing) are checked against the layout
// index of every position.  Half the circuits plan DENSE ops on register
// bits in place (the complex64 option).  This pins the planner's bookkeeping on the
// CPU; the GPU parity tests pin the kernels against the oracle.
//
// Build: g++ -O1 -std=c++17 -I<include> -I<csrc> -I<cuda include>
//        planner_emulator.cpp -L<pkg> -lqtask
// Prints "OK <passes> <ops>" and exits 0, or prints the first mismatch and
// exits 1.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "qt_internal.h"

using namespace qt;
using cd = std::complex<double>;

static cd entry(const DevOp& o, int k) { return cd(o.m.d[2 * k], o.m.d[2 * k + 1]); }

// ---------------------------------------------------------------- reference
static void apply_reference(const DevOp& o, std::vector<cd>& T, int tb, uint64_t base) {
    if ((base & o.cm_glob) != o.cm_glob) return;
    const uint32_t n = 1u << tb;
    auto cond = [&](uint32_t j) { return (j & o.cm_tile) == o.cm_tile; };
    switch (o.kind) {
        case OP_DENSE: case OP_REAL: case OP_IREAL: case OP_X: case OP_ANTI: {
            const uint32_t tbit = 1u << o.b0;
            for (uint32_t j = 0; j < n; ++j) {
                if ((j & tbit) || !cond(j)) continue;
                const cd a = T[j], b = T[j | tbit];
                if (o.kind == OP_X) {
                    T[j] = b;
                    T[j | tbit] = a;
                } else if (o.kind == OP_ANTI) {
                    T[j] = entry(o, 0) * b;
                    T[j | tbit] = entry(o, 1) * a;
                } else {
                    T[j] = entry(o, 0) * a + entry(o, 1) * b;
                    T[j | tbit] = entry(o, 2) * a + entry(o, 3) * b;
                }
            }
            break;
        }
        case OP_SWAP: {
            const uint32_t m0 = 1u << o.b0, m1 = 1u << o.b1;
            for (uint32_t j = 0; j < n; ++j)
                if ((j & m0) && !(j & m1) && cond(j)) std::swap(T[j], T[j ^ (m0 | m1)]);
            break;
        }
        case OP_DIAG: {
            for (uint32_t j = 0; j < n; ++j) {
                if (!cond(j)) continue;
                const int bit = o.b0 < 0 ? int((base >> o.gq) & 1u) : int((j >> o.b0) & 1u);
                T[j] *= entry(o, bit);
            }
            break;
        }
        case OP_PHASE: {
            cd f = entry(o, 0);
            if (o.sub == PH_NEG) f = -1.0;
            else if (o.sub == PH_POS_I) f = cd(0.0, 1.0);
            else if (o.sub == PH_NEG_I) f = cd(0.0, -1.0);
            for (uint32_t j = 0; j < n; ++j)
                if (cond(j)) T[j] *= f;
            break;
        }
        default:
            break;
    }
}

// ----------------------------------------------------------------- planned
struct Phys {
    int nreg, nwarp, R, W;
    std::vector<cd> v;  // slot (lane, r, w) -> lane + 32 * (r + R * w)
    cd& at(int lane, int r, int w) { return v[size_t(lane) + 32u * size_t(r + R * w)]; }
};

static uint32_t layout_index(const int8_t* lane, const int8_t* reg, const int8_t* warp, int nreg, int nwarp,
                             uint32_t flip, int l, int r, int w) {
    uint32_t j = 0;
    for (int i = 0; i < 5; ++i)
        if ((l >> i) & 1) j |= 1u << (lane ? lane[i] : i);
    for (int k = 0; k < nreg; ++k)
        if ((r >> k) & 1) j |= 1u << reg[k];
    for (int k = 0; k < nwarp; ++k)
        if ((w >> k) & 1) j |= 1u << warp[k];
    return j ^ flip;
}

// The kernel addresses register r of a thread as the amplitude index of the
// thread's tile index XOR the offsets of r's register bits (set_register_offsets);
// check that against the index of every (lane, register, warp) position, for
// the initial and the final layout.
static bool check_register_offsets(const DevPass& dp) {
    const uint32_t lowmask = (1u << dp.lt) - 1u;
    auto gidx = [&](uint32_t j) {
        uint64_t g = j & lowmask;
        for (int k = 0; k < dp.nh; ++k)
            if ((j >> (dp.lt + k)) & 1u) g |= uint64_t(1) << dp.h[k];
        return g;
    };
    int8_t reg0[8], warp0[8];
    for (int k = 0; k < dp.nreg; ++k) reg0[k] = int8_t(dp.layout[k]);
    for (int w = 0; w < dp.nwarp; ++w) warp0[w] = int8_t(dp.layout[dp.nreg + w]);
    for (int side = 0; side < 2; ++side) {
        const int8_t* ln = side ? dp.fin.lane : nullptr;
        const int8_t* rg = side ? dp.fin.reg : reg0;
        const int8_t* wp = side ? dp.fin.warp : warp0;
        const uint32_t flip = side ? dp.fin.flip : 0u;
        const uint64_t* off = side ? dp.rout : dp.rin;
        for (int w = 0; w < (1 << dp.nwarp); ++w)
            for (int l = 0; l < 32; ++l) {
                const uint64_t g0 = gidx(layout_index(ln, rg, wp, dp.nreg, dp.nwarp, flip, l, 0, w));
                for (int r = 0; r < (1 << dp.nreg); ++r) {
                    uint64_t got = g0;
                    for (int k = 0; k < dp.nreg; ++k)
                        if ((r >> k) & 1) got ^= off[k];
                    if (got != gidx(layout_index(ln, rg, wp, dp.nreg, dp.nwarp, flip, l, r, w))) return false;
                }
            }
    }
    return true;
}

static long g_groups = 0;  // merged phase groups seen
static long g_blocks = 0;  // tensor-core blocks seen
static long g_dense_k = 0;  // DENSE ops planned in place on a register bit above 0

static void run_planned(const std::vector<DevOp>& ops, const DevPass& dp, std::vector<cd>& T, uint64_t base,
                        const std::vector<Block>* blocks = nullptr) {
    Phys P{dp.nreg, dp.nwarp, 1 << dp.nreg, 1 << dp.nwarp, {}};
    P.v.assign(size_t(32) * P.R * P.W, 0.0);
    int8_t reg0[8], warp0[8];
    for (int k = 0; k < dp.nreg; ++k) reg0[k] = int8_t(dp.layout[k]);
    for (int w = 0; w < dp.nwarp; ++w) warp0[w] = int8_t(dp.layout[dp.nreg + w]);
    for (int w = 0; w < P.W; ++w)
        for (int r = 0; r < P.R; ++r)
            for (int l = 0; l < 32; ++l) P.at(l, r, w) = T[layout_index(nullptr, reg0, warp0, P.nreg, P.nwarp, 0, l, r, w)];
    for (size_t oi = 0; oi < ops.size(); ++oi) {
        const DevOp& o = ops[oi];
        const RegHdr& h = o.rh;
        if (h.code == RC_PH_GROUP) {
            // merged phases: per thread, the product of each step's terms whose
            // conditions hold, applied to the step's registers
            const int nt = o.b1;
            const size_t nslots = size_t((nt + kTermsPerSlot - 1) / kTermsPerSlot);
            if (nt < 1 || (oi % kOpChunk) + 1 + nslots > size_t(kOpChunk) || oi + nslots >= ops.size()) {
                std::printf("malformed phase group at op %zu\n", oi);
                std::exit(1);
            }
            const PhTerm* tm = reinterpret_cast<const PhTerm*>(&ops[oi + 1]);
            for (int w = 0; w < P.W; ++w) {
                for (int l = 0; l < 32; ++l) {
                    const uint32_t ptid = uint32_t(l) | (uint32_t(w) << 5);
                    for (int i = 0; i < nt;) {
                        cd f = 1.0;
                        bool go = false;
                        int mcls = 0, k = 0;
                        for (; i < nt; ++i) {
                            const PhTerm& t = tm[i];
                            if ((base & t.cm_glob) == t.cm_glob && ((ptid ^ t.cv_thr) & t.cm_thr) == t.cm_thr) {
                                f *= cd(t.f.d[0], t.f.d[1]);
                                go = true;
                            }
                            mcls = t.mcls;
                            k = t.k;
                            if (t.last) break;
                        }
                        ++i;
                        if (go)
                            for (int r = 0; r < P.R; ++r)
                                if (mcls == 0 || ((r >> k) & 1)) P.at(l, r, w) *= f;
                    }
                }
            }
            oi += nslots;
            ++g_groups;
            continue;
        }
        if (h.code == RC_MMA) {
            // the block on the tensor cores: gather the 128 x 32 operand through
            // the op's bit contributions, multiply by the block's matrix, and
            // scatter through the fixed layout that follows the op
            const BlockStage& bs = *reinterpret_cast<const BlockStage*>(&o.m);
            const Block& blk = blocks->at(size_t(bs.boff / kBlockBytes));
            std::vector<cd> Am(128 * 32), Dm(128 * 32, 0.0);
            for (int w = 0; w < P.W; ++w)
                for (int r = 0; r < P.R; ++r)
                    for (int l = 0; l < 32; ++l) {
                        uint32_t a = bs.a_flip;
                        for (int i = 0; i < 5; ++i)
                            if ((l >> i) & 1) a ^= bs.a_lane[i];
                        for (int k = 0; k < P.nreg; ++k)
                            if ((r >> k) & 1) a ^= bs.a_reg[k];
                        for (int k = 0; k < P.nwarp; ++k)
                            if ((w >> k) & 1) a ^= bs.a_warp[k];
                        // decode the swizzled operand-A byte offset into (row, block index)
                        const uint32_t m = ((a >> 10) & 15u) << 3 | ((a >> 7) & 7u);
                        const uint32_t kb = ((a >> 14) & 1u) << 4 | ((((a >> 4) & 7u) ^ (m & 7u)) << 1) | ((a >> 3) & 1u);
                        if (block_a_offset(m, kb) != a) {
                            std::printf("operand offset %u is not a (row, block index) position\n", a);
                            std::exit(1);
                        }
                        Am[m * 32 + kb] = P.at(l, r, w);
                    }
            for (int m = 0; m < 128; ++m)
                for (int jo = 0; jo < 32; ++jo)
                    for (int ji = 0; ji < 32; ++ji)
                        Dm[m * 32 + jo] += cd(blk.u[2 * (jo * 32 + ji)], blk.u[2 * (jo * 32 + ji) + 1]) * Am[m * 32 + ji];
            for (int w = 0; w < P.W; ++w)
                for (int r = 0; r < P.R; ++r)
                    for (int l = 0; l < 32; ++l) P.at(l, r, w) = Dm[(l | ((w & 3) << 5)) * 32 + (r | ((w >> 2) << 4))];
            ++g_blocks;
            continue;
        }
        if (h.code == RC_PERM) {
            TileLayout from;
            std::memcpy(&from, &o.m, sizeof from);
            std::vector<cd> L(T.size());
            for (int w = 0; w < P.W; ++w)
                for (int r = 0; r < P.R; ++r)
                    for (int l = 0; l < 32; ++l)
                        L[layout_index(from.lane, from.reg, from.warp, P.nreg, P.nwarp, from.flip, l, r, w)] = P.at(l, r, w);
            for (int w = 0; w < P.W; ++w)
                for (int r = 0; r < P.R; ++r)
                    for (int l = 0; l < 32; ++l)
                        P.at(l, r, w) = L[layout_index(nullptr, o.perm, o.perm + P.nreg, P.nreg, P.nwarp, 0, l, r, w)];
            continue;
        }
        if (h.ren > 0) {
            const int K = h.ren;
            for (int w = 0; w < P.W; ++w)
                for (int l = 0; l < 32; ++l)
                    for (int r = 0; r < P.R; ++r)
                        if ((r & 1) && !((r >> K) & 1)) std::swap(P.at(l, r, w), P.at(l, r ^ (1 | (1 << K)), w));
        }
        // DENSE, REAL, ANTI, IREAL and DIAG ops carry no conditions: the
        // kernel tests none for them
        const bool unconditioned = (h.code >= RC_DENSE_R && h.code <= RC_IREAL_L) ||
                                   (h.code >= RC_DIAG_G && h.code <= RC_DIAG_R);
        if (unconditioned && (o.cm_glob != 0 || h.cm_thr != 0 || h.cm_reg != 0)) {
            std::printf("op with code %d carries conditions\n", int(h.code));
            std::exit(1);
        }
        if ((base & o.cm_glob) != o.cm_glob) continue;
        if (h.code == RC_DENSE_R && h.b > 0) ++g_dense_k;
        const uint32_t cmr = h.cm_reg, cvr = h.cv_reg;
        auto rcond = [&](int r) { return ((uint32_t(r) ^ cvr) & cmr) == cmr; };
        Phys Q = P;  // values before the op (partners read from here)
        for (int w = 0; w < P.W; ++w) {
            for (int l = 0; l < 32; ++l) {
                const uint32_t ptid = uint32_t(l) | (uint32_t(w) << 5);
                const bool thr_ok = ((ptid ^ h.cv_thr) & h.cm_thr) == h.cm_thr;
                const int code = h.code;
                if (code == RC_DENSE_R || code == RC_REAL_R || code == RC_IREAL_R) {
                    const int K = code == RC_DENSE_R ? h.b : 0;  // DENSE may pair across register bit b
                    for (int r = 0; r < P.R; ++r) {
                        if ((r >> K) & 1) continue;
                        const int r1 = r | (1 << K);
                        const cd a = Q.at(l, r, w), b = Q.at(l, r1, w);
                        P.at(l, r, w) = entry(o, 0) * a + entry(o, 1) * b;
                        P.at(l, r1, w) = entry(o, 2) * a + entry(o, 3) * b;
                    }
                } else if (code == RC_DENSE_L || code == RC_REAL_L || code == RC_IREAL_L) {
                    const int hi = (l >> h.a) & 1, pl = l ^ (1 << h.a);
                    for (int r = 0; r < P.R; ++r) {
                        const cd own = Q.at(l, r, w), par = Q.at(pl, r, w);
                        P.at(l, r, w) = hi ? entry(o, 3) * own + entry(o, 2) * par : entry(o, 0) * own + entry(o, 1) * par;
                    }
                } else if (code == RC_ANTI_R) {
                    for (int r = 0; r < P.R; r += 2) {
                        const cd a = Q.at(l, r, w), b = Q.at(l, r + 1, w);
                        P.at(l, r, w) = entry(o, 0) * b;
                        P.at(l, r + 1, w) = entry(o, 1) * a;
                    }
                } else if (code == RC_ANTI_L) {
                    const int hi = (l >> h.a) & 1, pl = l ^ (1 << h.a);
                    for (int r = 0; r < P.R; ++r) P.at(l, r, w) = entry(o, hi) * Q.at(pl, r, w);
                } else if (code == RC_X_R) {
                    for (int r = 0; r < P.R; r += 2)
                        if (thr_ok && rcond(r)) std::swap(P.at(l, r, w), P.at(l, r + 1, w));
                } else if (code == RC_X_L) {
                    const int pl = l ^ (1 << h.a);
                    for (int r = 0; r < P.R; ++r)
                        if (thr_ok && rcond(r)) P.at(l, r, w) = Q.at(pl, r, w);
                } else if (code == RC_SWAP_RR) {
                    const int K0 = h.a, K1 = h.b;
                    for (int r = 0; r < P.R; ++r)
                        if (((r >> K0) & 1) && !((r >> K1) & 1) && thr_ok && rcond(r))
                            std::swap(P.at(l, r, w), P.at(l, r ^ ((1 << K0) | (1 << K1)), w));
                } else if (code == RC_SWAP_LR) {
                    const int b = h.a, K = h.b, pl = l ^ (1 << b);
                    const bool lb = (l >> b) & 1;
                    for (int r = 0; r < P.R; ++r) {
                        if (r & (1 << K)) continue;
                        const int r1 = r | (1 << K);
                        if (!(thr_ok && rcond(r))) continue;
                        if (lb) P.at(l, r, w) = Q.at(pl, r1, w);
                        else P.at(l, r1, w) = Q.at(pl, r, w);
                    }
                } else if (code == RC_SWAP_LL) {
                    const int mask = (1 << h.a) | (1 << h.b), pl = l ^ mask;
                    const bool differ = ((l >> h.a) ^ (l >> h.b)) & 1;
                    for (int r = 0; r < P.R; ++r)
                        if (differ && thr_ok && rcond(r)) P.at(l, r, w) = Q.at(pl, r, w);
                } else if (code == RC_DIAG_G || code == RC_DIAG_T) {
                    const int bit = code == RC_DIAG_G ? int((base >> h.a) & 1u) : int((ptid >> h.a) & 1u);
                    for (int r = 0; r < P.R; ++r) P.at(l, r, w) *= entry(o, bit);
                } else if (code == RC_DIAG_R) {
                    for (int r = 0; r < P.R; ++r) P.at(l, r, w) *= entry(o, (r >> h.a) & 1);
                } else if (code >= RC_PH_NEG && code <= RC_PH_GEN) {
                    if (!thr_ok) continue;
                    cd f = entry(o, 0);
                    if (code == RC_PH_NEG) f = -1.0;
                    else if (code == RC_PH_POS_I) f = cd(0.0, 1.0);
                    else if (code == RC_PH_NEG_I) f = cd(0.0, -1.0);
                    for (int r = 0; r < P.R; ++r) {
                        const bool q = h.mcls == 0 ? true : h.mcls == 1 ? bool((r >> h.a) & 1) : rcond(r);
                        if (q) P.at(l, r, w) *= f;
                    }
                }
            }
        }
    }
    for (int w = 0; w < P.W; ++w)
        for (int r = 0; r < P.R; ++r)
            for (int l = 0; l < 32; ++l)
                T[layout_index(dp.fin.lane, dp.fin.reg, dp.fin.warp, P.nreg, P.nwarp, dp.fin.flip, l, r, w)] = P.at(l, r, w);
}

int main(int argc, char** argv) {
    const int ncirc = argc > 1 ? atoi(argv[1]) : 40;
    std::mt19937_64 rng(20251204);
    std::uniform_real_distribution<double> U(-1.0, 1.0), ang(0.0, 6.283185307179586);
    long npasses = 0, nops = 0;
    for (int ci = 0; ci < ncirc; ++ci) {
        const int n = 11 + ci % 4;
        const int th = 3 + ci % 3;
        qt_circuit* c = nullptr;
        if (qt_create(n, QT_C128, n, &c) != QT_OK) return 2;
        qt_set_option(c, "tile_high", th);
        qt_set_option(c, "merge", ci % 2);
        const int ngates = 120 + 20 * (ci % 5);
        const bool ladder = ci % 5 == 4;  // QFT-like: H then controlled phases (runs of phases)
        for (int gi = 0; gi < ngates; ++gi) {
            qt_insert_level(c, gi);
            qt_gate g{};
            if (ladder) {
                const int j = (gi / n) % n, m = gi % n;
                if (m == j) {
                    g.kind = QT_H;
                    g.ntarget = 1;
                    g.target[0] = j;
                } else {
                    g.kind = (gi % 7 == 0) ? QT_CZ : QT_CP;
                    g.ntarget = 1;
                    g.target[0] = j;
                    g.ncontrol = 1;
                    g.control[0] = m;
                    g.theta[0] = ang(rng);
                }
                qt_gate_id id;
                if (qt_insert_gate(c, gi, &g, &id) != QT_OK) return 3;
                continue;
            }
            // weight permutations and phases: they exercise relabels and conditions
            static const int pool[] = {QT_H, QT_X, QT_X, QT_Y, QT_Z, QT_S, QT_SDG, QT_T, QT_RX, QT_RX, QT_RY, QT_RZ,
                                       QT_U3, QT_CNOT, QT_CNOT, QT_CZ, QT_SWAP, QT_SWAP, QT_CCX, QT_CP};
            g.kind = pool[rng() % (sizeof pool / sizeof pool[0])];
            const int nt = g.kind == QT_SWAP ? 2 : 1;
            const int nc = g.kind == QT_CCX ? 2 : (g.kind == QT_CNOT || g.kind == QT_CZ || g.kind == QT_CP) ? 1 : 0;
            int q[3];
            for (int k = 0; k < nt + nc; ++k) {
                bool fresh;
                do {
                    q[k] = int(rng() % uint64_t(n));
                    fresh = true;
                    for (int m = 0; m < k; ++m) fresh = fresh && q[m] != q[k];
                } while (!fresh);
            }
            g.ntarget = nt;
            g.ncontrol = nc;
            for (int k = 0; k < nt; ++k) g.target[k] = q[k];
            for (int k = 0; k < nc; ++k) g.control[k] = q[nt + k];
            for (int k = 0; k < 3; ++k) g.theta[k] = ang(rng);
            qt_gate_id id;
            if (qt_insert_gate(c, gi, &g, &id) != QT_OK) return 3;
        }
        std::vector<Pass> passes;
        int dtype = 0, nn = 0;
        circuit_plan_whole(c, &passes, &dtype, &nn);
        for (const Pass& ps : passes) {
            std::vector<DevOp> ops;
            for (const HostOp& ho : ps.ops) ops.push_back(encode_device_op(dtype, ps, ho));
            const int tb = ps.lt + ps.nh;
            if (tb < 7) continue;  // the shared-memory kernel: no register layout
            for (int reorder = 0; reorder < 2; ++reorder) {
                DevPass dp;
                std::memset(&dp, 0, sizeof dp);
                dp.lt = ps.lt;
                dp.nh = ps.nh;
                std::vector<DevOp> planned = ops;
                plan_register_layout(&dp, &planned, 16, reorder != 0, true, (ci & 1) != 0);
                for (int h = 0; h < ps.nh; ++h) dp.h[h] = ps.h[h];
                set_register_offsets(&dp);
                if (!check_register_offsets(dp)) {
                    std::printf("register offsets disagree with the layout (circuit %d)\n", ci);
                    return 1;
                }
                for (int trial = 0; trial < 2; ++trial) {
                    const uint64_t base = rng();
                    std::vector<cd> T(size_t(1) << tb);
                    for (cd& v : T) v = cd(U(rng), U(rng));
                    std::vector<cd> ref = T, got = T;
                    for (const DevOp& o : ops) apply_reference(o, ref, tb, base);
                    run_planned(planned, dp, got, base);
                    double err = 0.0;
                    for (size_t j = 0; j < T.size(); ++j) err = std::max(err, std::abs(ref[j] - got[j]));
                    if (!(err <= 1e-12)) {
                        std::printf("MISMATCH circuit %d pass of %zu ops tb %d reorder %d: max err %.3e\n", ci,
                                    ops.size(), tb, reorder, err);
                        return 1;
                    }
                }
                nops += long(planned.size());
            }
            ++npasses;
        }
        qt_destroy(c);
    }
    if (g_groups == 0) {
        std::printf("no merged phase group was planned\n");
        return 1;
    }
    // Tensor-core blocks (complex64 tiles of 12 qubits: 7 low, 5 high): the
    // passes planned with and without blocks cover the same gates; the
    // unfused ops applied directly must equal the planned ops with the
    // blocks' FP64 matrices.
    long nblk_passes = 0;
    for (int ci = 0; ci < ncirc; ++ci) {
        const int n = 12 + ci % 3;
        std::vector<qt_gate> gates;
        static const int pool[] = {QT_H, QT_U3, QT_U3, QT_RX, QT_RY, QT_RZ, QT_T, QT_X, QT_Y, QT_CNOT, QT_CZ, QT_CP,
                                   QT_SWAP, QT_CCX};
        const int ngates = 150 + 10 * (ci % 4);
        for (int gi = 0; gi < ngates; ++gi) {
            qt_gate g{};
            g.kind = pool[rng() % (sizeof pool / sizeof pool[0])];
            const int nt = g.kind == QT_SWAP ? 2 : 1;
            const int nc = g.kind == QT_CCX ? 2 : (g.kind == QT_CNOT || g.kind == QT_CZ || g.kind == QT_CP) ? 1 : 0;
            // qubits mostly from a window of 6, so that runs on five qubits form
            const int lo = int(rng() % uint64_t(n - 5));
            int q[3];
            for (int k = 0; k < nt + nc; ++k) {
                bool fresh;
                do {
                    q[k] = (rng() % 4 == 0) ? int(rng() % uint64_t(n)) : lo + int(rng() % 6);
                    fresh = true;
                    for (int m = 0; m < k; ++m) fresh = fresh && q[m] != q[k];
                } while (!fresh);
            }
            g.ntarget = nt;
            g.ncontrol = nc;
            for (int k = 0; k < nt; ++k) g.target[k] = q[k];
            for (int k = 0; k < nc; ++k) g.control[k] = q[nt + k];
            for (int k = 0; k < 3; ++k) g.theta[k] = ang(rng);
            gates.push_back(g);
        }
        std::vector<const qt_gate*> gl;
        for (const qt_gate& g : gates) gl.push_back(&g);
        PlanParams pp;
        pp.n = n;
        pp.p = n - 2;  // tiles reach into the partition index: coupled partitions
        pp.lt = 7;
        pp.nh_max = 5;
        pp.fusion = true;
        pp.merge = ci % 2 == 0;
        SegPlan plain = plan_segment(gl, pp);
        pp.tc_blocks = true;
        pp.tc_threshold = ci % 3 == 0 ? 0.0 : 2.0;
        SegPlan fused = plan_segment(gl, pp);
        if (plain.passes.size() != fused.passes.size()) {
            std::printf("blocks changed the pass partition\n");
            return 1;
        }
        for (size_t pi = 0; pi < fused.passes.size(); ++pi) {
            const Pass& pr = plain.passes[pi];
            const Pass& pf = fused.passes[pi];
            const int tb = pf.lt + pf.nh;
            if (tb != 12 || pf.blocks.empty()) continue;
            std::vector<DevOp> ref_ops;
            for (const HostOp& ho : pr.ops) ref_ops.push_back(encode_device_op(QT_C128, pr, ho));
            std::vector<float> blkbuf;
            std::vector<DevOp> ops;
            for (const HostOp& ho : pf.ops) ops.push_back(encode_device_op(QT_C128, pf, ho, &blkbuf));
            for (int reorder = 0; reorder < 2; ++reorder) {
                DevPass dp;
                std::memset(&dp, 0, sizeof dp);
                dp.lt = pf.lt;
                dp.nh = pf.nh;
                std::vector<DevOp> planned = ops;
                plan_register_layout(&dp, &planned, 16, reorder != 0, true, true);
                if (!dp.mma || dp.nreg != 4 || dp.nwarp != 3) {
                    std::printf("a pass with blocks was not planned for the tensor-core kernel\n");
                    return 1;
                }
                const uint64_t base = rng();
                std::vector<cd> T(size_t(1) << tb);
                for (cd& v : T) v = cd(U(rng), U(rng));
                std::vector<cd> ref = T, got = T;
                for (const DevOp& o : ref_ops) apply_reference(o, ref, tb, base);
                run_planned(planned, dp, got, base, &pf.blocks);
                double err = 0.0;
                for (size_t j = 0; j < T.size(); ++j) err = std::max(err, std::abs(ref[j] - got[j]));
                if (!(err <= 1e-12)) {
                    std::printf("MISMATCH (blocks) circuit %d pass %zu, %zu ops, %zu blocks, reorder %d: max err %.3e\n",
                                ci, pi, pf.ops.size(), pf.blocks.size(), reorder, err);
                    return 1;
                }
            }
            ++nblk_passes;
        }
    }
    if (g_dense_k == 0) {
        std::printf("no DENSE op was planned in place on a register bit\n");
        return 1;
    }
    if (g_blocks == 0) {
        std::printf("no tensor-core block was planned\n");
        return 1;
    }
    std::printf("OK %ld %ld %ld %ld %ld\n", npasses, nops, g_groups, nblk_passes, g_blocks);
    return 0;
}
