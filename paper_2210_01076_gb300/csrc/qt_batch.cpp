// qt_batch.cpp -- many small circuits in one persistent launch (C ABI
// qt_batch_*).
//
// Small circuits (10-20 qubits) cannot fill a GB300 one at a time: a pass
// over 2^15 amplitudes is a handful of CTAs.  A batch plans every circuit as
// one segment, lays their states out in one device arena, numbers the tiles
// of all passes in wavefront order, and runs them all in one persistent
// launch (qt_pass_reg.cu, k_batch) in which a tile waits only for the
// previous pass of its own circuit.  The launch, the arena initialisation to
// |0...0> and the uploads are captured once in a CUDA graph and replayed
// while the circuits keep their structure -- parameter edits (a rotation
// angle changed) only rewrite the op matrices the graph uploads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "qt_internal.h"

using namespace qt;

struct qt_batch {
    std::vector<qt_circuit*> circs;
    int dtype = -1;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void* arena = nullptr;
    uint64_t arena_amps = 0;
    std::vector<uint64_t> offsets;
    std::vector<int> ns;
    std::vector<int64_t> gates;
    BatchPass* d_passes = nullptr;
    DevOp* d_ops = nullptr;
    uint32_t* d_sync = nullptr;  // [0] = head, [1..] = pass counters
    int* d_err = nullptr;
    uint64_t* d_firsts = nullptr;
    BatchPass* h_passes = nullptr;
    DevOp* h_ops = nullptr;
    int* h_err = nullptr;
    size_t cap_passes = 0, cap_ops = 0, cap_sync = 0;
    int npasses = 0, nops = 0;
    uint32_t total_items = 0;
    size_t smem = 0;
    std::vector<uint8_t> signature;  // structure of the last run (everything but matrix values)
    bool ran_direct = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
};

namespace {

qt_status bfail(qt_batch* b, qt_status s, const std::string& m) {
    if (b) b->err = m;
    set_thread_error(m);
    return s;
}

void free_graph(qt_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

template <class T>
cudaError_t grow_dev(T** p, size_t* cap, size_t need) {
    if (need <= *cap) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), need * sizeof(T));
    if (e == cudaSuccess) *cap = need;
    return e;
}

template <class T>
cudaError_t grow_pinned(T** p, size_t need, size_t old) {
    if (need <= old) return cudaSuccess;
    cudaFreeHost(*p);
    *p = nullptr;
    return cudaMallocHost(reinterpret_cast<void**>(p), need * sizeof(T));
}

// Enqueue one run on b->stream (used directly or under stream capture).
cudaError_t enqueue(qt_batch* b) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_ops, b->h_ops, sizeof(DevOp) * std::max(b->nops, 1), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(b->d_passes, b->h_passes, sizeof(BatchPass) * std::max(b->npasses, 1),
                             cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(b->d_sync, 0, sizeof(uint32_t) * (size_t(b->npasses) + 1), b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream)) != cudaSuccess) return e;
    int rc = launch_batch_init(b->dtype, b->arena, b->arena_amps, b->d_firsts, int(b->circs.size()), b->stream);
    if (rc) return cudaError_t(rc);
    rc = launch_batch(b->dtype, b->arena, b->d_passes, b->npasses, b->d_ops, b->total_items, b->d_sync,
                      b->d_sync + 1, b->d_err, b->smem, b->stream);
    if (rc) return cudaError_t(rc);
    return cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
}

}  // namespace

extern "C" {

qt_status qt_batch_create(qt_circuit* const* circuits, int32_t count, qt_batch** out) {
    if (!out || !circuits || count < 1) return bfail(nullptr, QT_ERR_ARG, "qt_batch_create: bad arguments");
    try {
        qt_batch* b = new qt_batch();
        for (int i = 0; i < count; ++i) {
            if (!circuits[i]) {
                delete b;
                return bfail(nullptr, QT_ERR_ARG, "qt_batch_create: NULL circuit");
            }
            b->circs.push_back(circuits[i]);
        }
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreate(&b->ev0)) != cudaSuccess || (e = cudaEventCreate(&b->ev1)) != cudaSuccess ||
            (e = cudaMalloc(reinterpret_cast<void**>(&b->d_err), sizeof(int))) != cudaSuccess ||
            (e = cudaMallocHost(reinterpret_cast<void**>(&b->h_err), sizeof(int))) != cudaSuccess) {
            qt_batch_destroy(b);
            return bfail(nullptr, QT_ERR_CUDA, std::string("qt_batch_create: ") + cudaGetErrorString(e));
        }
        *out = b;
        return QT_OK;
    } catch (...) {
        return bfail(nullptr, QT_ERR_OOM, "qt_batch_create: host allocation failed");
    }
}

qt_status qt_batch_destroy(qt_batch* b) {
    if (!b) return QT_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_graph(b);
    cudaFree(b->arena);
    cudaFree(b->d_passes);
    cudaFree(b->d_ops);
    cudaFree(b->d_sync);
    cudaFree(b->d_err);
    cudaFree(b->d_firsts);
    cudaFreeHost(b->h_passes);
    cudaFreeHost(b->h_ops);
    cudaFreeHost(b->h_err);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return QT_OK;
}

qt_status qt_batch_run(qt_batch* b, qt_batch_stats* stats) {
    if (!b) return QT_ERR_ARG;
    try {
        // ---- plan every circuit as one segment
        const int nc = int(b->circs.size());
        std::vector<std::vector<Pass>> plans(nc);
        std::vector<int> ns(nc), dts(nc);
        std::vector<int64_t> gates(nc, 0);
        for (int c = 0; c < nc; ++c) {
            circuit_plan_whole(b->circs[c], &plans[c], &dts[c], &ns[c]);
            for (const Pass& ps : plans[c]) gates[c] += ps.ngates;
            if (dts[c] != dts[0]) return bfail(b, QT_ERR_ARG, "qt_batch_run: all circuits must share a dtype");
        }
        const int dtype = dts[0];
        // ---- encode passes (per circuit, in order)
        struct Enc {
            DevPass dp;
            std::vector<DevOp> ops;
            uint32_t ntiles;
        };
        std::vector<std::vector<Enc>> enc(nc);
        size_t maxp = 0, smem = 0;
        for (int c = 0; c < nc; ++c) {
            for (const Pass& ps : plans[c]) {
                Enc en;
                DevPass& dp = en.dp;
                std::memset(&dp, 0, sizeof dp);
                dp.p = ns[c];
                dp.lt = ps.lt;
                dp.nh = ps.nh;
                dp.nins = ps.nh;
                for (int h = 0; h < ps.nh; ++h) dp.h[h] = dp.ins[h] = ps.h[h];
                dp.tpg_log2 = ns[c] - ps.lt - ps.nh;
                dp.M = 0;
                dp.npart_log2 = 0;
                for (const HostOp& o : ps.ops) en.ops.push_back(encode_device_op(dtype, ps, o));
                // batches run the kernel without merged phase groups
                // (in-place DENSE on register bits measured 0.9 % slower in the batched launch)
                plan_register_layout(&dp, &en.ops, int(bytes_per_amp(dtype)), true, false, false);
                if (dp.reg_kernel) set_register_offsets(&dp);
                dp.nops = int32_t(en.ops.size());
                if (!dp.reg_kernel || dp.nwarp != 3 || dp.nreg < 2 || dp.nreg > 4)
                    return bfail(b, QT_ERR_ARG,
                                 "qt_batch_run: circuits need tiles of 2^10 to 2^12 amplitudes (10 or more qubits)");
                // k_batch keeps a tile in at most 64 KB of shared memory and
                // instantiates 2^12-amplitude tiles for 8-byte amplitudes only
                if (dp.nreg == 4 && bytes_per_amp(dtype) != 8)
                    return bfail(b, QT_ERR_ARG,
                                 "qt_batch_run: 16-byte amplitudes need tiles of at most 2^11 amplitudes "
                                 "(set tile_high <= 5)");
                en.ntiles = 1u << dp.tpg_log2;
                smem = std::max(smem, bytes_per_amp(dtype) << (dp.lt + dp.nh));
                enc[c].push_back(std::move(en));
            }
            maxp = std::max(maxp, enc[c].size());
        }
        // ---- wavefront order, signature
        std::vector<BatchPass> hp;
        std::vector<DevOp> hops;
        std::vector<uint8_t> sig;
        auto put = [&](const void* p, size_t nbytes) {
            const uint8_t* q = static_cast<const uint8_t*>(p);
            sig.insert(sig.end(), q, q + nbytes);
        };
        std::vector<uint64_t> offsets(nc);
        uint64_t amps = 0;
        for (int c = 0; c < nc; ++c) {
            offsets[c] = amps;
            amps += std::max<uint64_t>(uint64_t(1) << ns[c], 32);  // 512-byte aligned starts
        }
        std::vector<int> prev_counter(nc, -1);
        std::vector<uint32_t> prev_tiles(nc, 0);
        uint32_t items = 0;
        for (size_t i = 0; i < maxp; ++i) {
            for (int c = 0; c < nc; ++c) {
                if (i >= enc[c].size()) continue;
                Enc& en = enc[c][i];
                BatchPass bp;
                std::memset(&bp, 0, sizeof bp);
                bp.dp = en.dp;
                bp.dp.op_offset = int64_t(hops.size());
                bp.state_off = offsets[c];
                bp.first_item = items;
                bp.ntiles = en.ntiles;
                bp.dep = prev_counter[c];
                bp.dep_need = prev_tiles[c];
                bp.counter = int32_t(hp.size());
                prev_counter[c] = bp.counter;
                prev_tiles[c] = en.ntiles;
                items += en.ntiles;
                hp.push_back(bp);
                put(&bp, sizeof bp);
                for (const DevOp& o : en.ops) {
                    DevOp s = o;
                    std::memset(&s.m, 0, sizeof s.m);  // matrices may change without a new graph
                    put(&s, sizeof s);
                    hops.push_back(o);
                }
            }
        }
        put(&amps, sizeof amps);
        // ---- device buffers and upload staging
        const bool same = (sig == b->signature) && b->dtype == dtype;
        cudaError_t e;
        if (!same) {
            free_graph(b);
            b->ran_direct = false;
            cudaStreamSynchronize(b->stream);
            if (amps != b->arena_amps || dtype != b->dtype) {
                cudaFree(b->arena);
                b->arena = nullptr;
                if ((e = cudaMalloc(&b->arena, amps * bytes_per_amp(dtype))) != cudaSuccess) {
                    cudaGetLastError();
                    b->arena_amps = 0;
                    return bfail(b, QT_ERR_OOM, "qt_batch_run: arena allocation failed");
                }
                b->arena_amps = amps;
            }
            cudaFree(b->d_firsts);
            b->d_firsts = nullptr;
            if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_firsts), sizeof(uint64_t) * nc)) != cudaSuccess)
                return bfail(b, QT_ERR_OOM, "qt_batch_run: allocation failed");
            if ((e = cudaMemcpy(b->d_firsts, offsets.data(), sizeof(uint64_t) * nc, cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return bfail(b, QT_ERR_CUDA, "qt_batch_run: upload failed");
            const size_t old_p = b->cap_passes, old_o = b->cap_ops;
            if (grow_dev(&b->d_passes, &b->cap_passes, std::max<size_t>(hp.size(), 1)) != cudaSuccess ||
                grow_dev(&b->d_ops, &b->cap_ops, std::max<size_t>(hops.size(), 1)) != cudaSuccess ||
                grow_dev(&b->d_sync, &b->cap_sync, hp.size() + 1) != cudaSuccess)
                return bfail(b, QT_ERR_OOM, "qt_batch_run: allocation failed");
            if (grow_pinned(&b->h_passes, b->cap_passes, old_p) != cudaSuccess ||
                grow_pinned(&b->h_ops, b->cap_ops, old_o) != cudaSuccess)
                return bfail(b, QT_ERR_OOM, "qt_batch_run: pinned allocation failed");
            b->signature = sig;
            b->dtype = dtype;
        }
        std::memcpy(b->h_passes, hp.data(), sizeof(BatchPass) * hp.size());
        std::memcpy(b->h_ops, hops.data(), sizeof(DevOp) * hops.size());
        b->npasses = int(hp.size());
        b->nops = int(hops.size());
        b->total_items = items;
        b->smem = smem;
        b->offsets = offsets;
        b->ns = ns;
        b->gates = gates;
        // ---- run: directly the first time (kernel attributes are set
        // outside any capture), then from a captured graph
        bool replayed = false;
        if ((e = cudaEventRecord(b->ev0, b->stream)) != cudaSuccess) return bfail(b, QT_ERR_CUDA, "event");
        if (!b->ran_direct) {
            if ((e = enqueue(b)) != cudaSuccess) return bfail(b, QT_ERR_CUDA, cudaGetErrorString(e));
            b->ran_direct = true;
        } else {
            if (!b->gexec) {
                if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                    return bfail(b, QT_ERR_CUDA, cudaGetErrorString(e));
                cudaError_t ce = enqueue(b);
                e = cudaStreamEndCapture(b->stream, &b->graph);
                if (ce != cudaSuccess || e != cudaSuccess)
                    return bfail(b, QT_ERR_CUDA, cudaGetErrorString(ce != cudaSuccess ? ce : e));
                if ((e = cudaGraphInstantiate(&b->gexec, b->graph, 0)) != cudaSuccess)
                    return bfail(b, QT_ERR_CUDA, cudaGetErrorString(e));
            } else {
                replayed = true;
            }
            if ((e = cudaGraphLaunch(b->gexec, b->stream)) != cudaSuccess)
                return bfail(b, QT_ERR_CUDA, cudaGetErrorString(e));
        }
        if ((e = cudaEventRecord(b->ev1, b->stream)) != cudaSuccess) return bfail(b, QT_ERR_CUDA, "event");
        if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bfail(b, QT_ERR_CUDA, cudaGetErrorString(e));
        if (*b->h_err == 2) return bfail(b, QT_ERR_ARG, "qt_batch_run: a tile shape the batch kernel does not support");
        if (*b->h_err) return bfail(b, QT_ERR_TIMEOUT, "qt_batch_run: a bounded wait between passes expired");
        if (stats) {
            std::memset(stats, 0, sizeof *stats);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, b->ev0, b->ev1);
            stats->gpu_ms = ms;
            stats->circuits = nc;
            stats->passes = b->npasses;
            stats->tiles = int32_t(items);
            stats->graph_replayed = replayed ? 1 : 0;
            for (int c = 0; c < nc; ++c) stats->amp_updates += uint64_t(gates[c]) << ns[c];
        }
        return QT_OK;
    } catch (const std::exception& ex) {
        return bfail(b, QT_ERR_ARG, std::string("qt_batch_run: ") + ex.what());
    } catch (...) {
        return bfail(b, QT_ERR_OOM, "qt_batch_run: host allocation failed");
    }
}

qt_status qt_batch_read_amplitudes(const qt_batch* cb, int32_t index, uint64_t first, uint64_t count,
                                   void* host_dst) {
    qt_batch* b = const_cast<qt_batch*>(cb);
    if (!b || (count && !host_dst)) return QT_ERR_ARG;
    if (index < 0 || index >= int32_t(b->ns.size())) return bfail(b, QT_ERR_RANGE, "no such circuit in the last run");
    const uint64_t N = uint64_t(1) << b->ns[index];
    if (first > N || count > N - first) return bfail(b, QT_ERR_RANGE, "amplitude range");
    if (count == 0) return QT_OK;
    const size_t bpa = bytes_per_amp(b->dtype);
    const char* src = static_cast<const char*>(b->arena) + (b->offsets[index] + first) * bpa;
    cudaError_t e;
    if (b->dtype != QT_C128_DF) {
        e = cudaMemcpy(host_dst, src, count * bpa, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? QT_OK : bfail(b, QT_ERR_CUDA, cudaGetErrorString(e));
    }
    void* tmp = nullptr;
    if ((e = cudaMalloc(&tmp, count * 16)) != cudaSuccess) return bfail(b, QT_ERR_OOM, "staging buffer");
    int rc = launch_read_convert(b->dtype, tmp, static_cast<const char*>(b->arena) + b->offsets[index] * bpa, first,
                                 count, b->stream);
    if (!rc) e = cudaMemcpyAsync(host_dst, tmp, count * 16, cudaMemcpyDeviceToHost, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (rc) return bfail(b, QT_ERR_CUDA, cudaGetErrorString(cudaError_t(rc)));
    return e == cudaSuccess ? QT_OK : bfail(b, QT_ERR_CUDA, cudaGetErrorString(e));
}

const char* qt_batch_last_error(const qt_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
