// batch.cu -- many independent problems advanced together: one time step of the whole batch is one
// CUDA graph. The MC legs of all problems run as one persistent work-queue launch (CTAs pull
// (problem, history range) chunks from a device queue, so uneven banks balance across the GPU);
// normalisation, the collided S_N-DG solves and the remaps of the problems follow as independent
// branches on a pool of streams. Each problem's results are those of stepping it alone: every
// kernel works on one problem's data, and all sums are order-free integers.
//
// Graph replay needs no host state change between steps: the step index and the point-set keys
// live in device memory, source iteration stops on a device flag (later iterations return at
// once), and the banks' double buffer is handled by two graphs, one per parity, replayed in turn.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "hyb_device.cuh"

namespace {

struct LegChunkH { int p; int pad; long long j0, j1; };

thread_local std::string g_batch_err;

}  // namespace

struct hyb_batch {
    std::vector<hyb_problem*> probs;
    int prec = 0;
    cudaStream_t s0 = nullptr;
    bool own_s0 = false;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> join_ev;
    cudaEvent_t fork_ev = nullptr, ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evl0 = nullptr, evl1 = nullptr;   // around the batched births and leg (external nodes in graphs)
    void* d_args[2] = {nullptr, nullptr};   // per parity: LegArgs of every problem
    size_t cap_probs = 0;                   // problems the per-problem buffers hold (grow-only)
    size_t cap_chunks = 0, cap_bchunks = 0; // chunk queue capacities (grow-only)
    void* d_chunks = nullptr;
    int nchunks = 0;
    void* d_bchunks = nullptr;              // birth chunks: (problem, [i0, i1) of its births)
    int nbchunks = 0;
    int* d_head = nullptr;                  // two queue heads: leg, births
    hyb::DevState* d_report = nullptr;      // per problem: a copy of its counters after the step
    hyb::DevState* h_report = nullptr;      // pinned
    uint32_t* d_V = nullptr;
    int ntab_max = 0;
    hyb_batch_tuning tune{256, 4096, 0, 8, 1, 0};
    std::vector<int> cur0;                  // bank parity of each problem when the batch was made
    std::vector<int> kmax;                  // source-iteration cap per problem inside the graph
    cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [parity][phase]
    std::vector<void*> phi_mid[2], old_mid[2];   // S_N buffer pointers between the phases
    int parity = 0;                         // graphs to replay next
    std::string err;
};

namespace {

hyb_status bfail(hyb_batch* b, hyb_status s, const std::string& m) {
    if (b) b->err = m; else g_batch_err = m;
    return s;
}

__global__ void report_kernel(const hyb::DevState* st, hyb::DevState* out) {
    const int i = threadIdx.x;
    const int n = (int)(sizeof(hyb::DevState) / sizeof(int));
    const int* src = (const int*)st;
    int* dst = (int*)out;
    for (int k = i; k < n; k += blockDim.x) dst[k] = src[k];
}

void drop_graphs(hyb_batch* b) {
    for (int q = 0; q < 2; ++q)
        for (int f = 0; f < 2; ++f)
            if (b->exec[q][f]) { cudaGraphExecDestroy(b->exec[q][f]); b->exec[q][f] = nullptr; }
}

hyb_status build_chunks(hyb_batch* b) {
    std::vector<LegChunkH> ch, bch;
    const long long C = std::max(32, b->tune.chunk);
    for (size_t i = 0; i < b->probs.size(); ++i) {
        hyb_problem* p = b->probs[i];
        const long long nsrc = p->has_src ? p->d.n_hist : 0;
        const long long N = p->bank_cap + nsrc;
        for (long long j = 0; j < std::max(N, 1LL); j += C) ch.push_back(LegChunkH{(int)i, 0, j, std::min(N, j + C)});
        for (long long j = 0; j < nsrc; j += C) bch.push_back(LegChunkH{(int)i, 0, j, std::min(nsrc, j + C)});
    }
    // interleave problems so that large banks do not end the queue alone
    std::stable_sort(ch.begin(), ch.end(), [](const LegChunkH& x, const LegChunkH& y) { return x.j0 < y.j0; });
    std::stable_sort(bch.begin(), bch.end(), [](const LegChunkH& x, const LegChunkH& y) { return x.j0 < y.j0; });
    auto ensure = [](void** d, size_t* cap, size_t need) {
        need = std::max<size_t>(need, 1);
        if (*cap >= need) return true;
        if (*d) cudaFree(*d);
        *d = nullptr;
        *cap = 0;
        if (cudaMalloc(d, need * sizeof(LegChunkH)) != cudaSuccess) return false;
        *cap = need;
        return true;
    };
    if (!ensure(&b->d_chunks, &b->cap_chunks, ch.size()) || !ensure(&b->d_bchunks, &b->cap_bchunks, bch.size()))
        return bfail(b, HYB_ENOMEM, "chunk queue allocation");
    if (cudaMemcpy(b->d_chunks, ch.data(), ch.size() * sizeof(LegChunkH), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!bch.empty() && cudaMemcpy(b->d_bchunks, bch.data(), bch.size() * sizeof(LegChunkH),
                                    cudaMemcpyHostToDevice) != cudaSuccess))
        return bfail(b, HYB_ECUDA, "chunk queue upload");
    b->nchunks = (int)ch.size();
    b->nbchunks = (int)bch.size();
    return HYB_OK;
}

// One phase of a batch step of parity q, issued on the batch streams (recorded into a graph by
// capture(), or run directly in eager mode). Phase 0: zero tallies and counters, the batched MC
// leg, then per problem normalisation and up to kmax source iterations (device stop). Phase 1: per
// problem the end of the collided solve, the remap and a copy of its counters. Problems whose
// iteration did not converge in phase 0 continue eagerly in between.
cudaError_t issue_phase(hyb_batch* b, int q, int phase) {
    const size_t n = b->probs.size();
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (phase == 0) {
        for (size_t i = 0; i < n; ++i) {
            hyb_problem* p = b->probs[i];
            const size_t nc = (size_t)p->ncells, acc = p->prec == HYB_FP64 ? 16 : 8;
            const size_t ncp = (size_t)p->tally_copies;
            ck(cudaMemsetAsync(p->acc_pre, 0, ncp * nc * acc, b->s0));
            ck(cudaMemsetAsync(p->acc_post, 0, ncp * nc * acc, b->s0));
            ck(cudaMemsetAsync(p->acc_mom, 0, ncp * 4 * nc * acc, b->s0));
            ck(cudaMemsetAsync(p->st, 0, offsetof(hyb::DevState, r_histories), b->s0));
            ck(cudaMemsetAsync(&p->st->status, 0, sizeof(int), b->s0));
        }
        ck(cudaMemsetAsync(b->d_head, 0, 2 * sizeof(int), b->s0));
        const int per_sm = b->tune.ctas_per_sm > 0 ? b->tune.ctas_per_sm
                                                   : hyb::leg_batch_ctas_per_sm(b->prec) * 256 / b->tune.block;
        const int grid = std::max(1, std::min(b->nchunks, sms * per_sm));
        // events around the births and the leg: external event nodes inside a captured graph (so
        // their times can be read after a replay), plain records when issued directly
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        ck(cudaStreamIsCapturing(b->s0, &cs));
        const bool capt = cs == cudaStreamCaptureStatusActive;
        ck(capt ? cudaEventRecordWithFlags(b->evl0, b->s0, cudaEventRecordExternal) : cudaEventRecord(b->evl0, b->s0));
        ck(hyb::launch_mc_leg_batch(b->prec, b->d_args[q], b->d_chunks, b->nchunks, b->d_head, b->d_V, b->ntab_max,
                                    grid, b->tune.block, b->s0, b->d_bchunks, b->nbchunks, b->d_head + 1));
        ck(capt ? cudaEventRecordWithFlags(b->evl1, b->s0, cudaEventRecordExternal) : cudaEventRecord(b->evl1, b->s0));
    }
    ck(cudaEventRecord(b->fork_ev, b->s0));
    for (auto s : b->pool) ck(cudaStreamWaitEvent(s, b->fork_ev, 0));
    for (size_t i = 0; i < n; ++i) {
        hyb_problem* p = b->probs[i];
        p->stream = b->pool[i % b->pool.size()];
        if (phase == 0) {
            ck(hyb::launch_leg_normalise(p));
            ck(hyb::sn_start(p));
            for (int k = 1; k <= b->kmax[i]; ++k) ck(hyb::sn_iteration(p, k == 1));
        } else {
            ck(hyb::sn_finish(p));
            ck(cudaMemsetAsync(&p->st->status, 0, sizeof(int), p->stream));
            ck(hyb::launch_remap(p));
        }
        report_kernel<<<1, 128, 0, p->stream>>>(p->st, b->d_report + i);
        ck(cudaGetLastError());
    }
    for (size_t j = 0; j < b->pool.size(); ++j) {
        ck(cudaEventRecord(b->join_ev[j], b->pool[j]));
        ck(cudaStreamWaitEvent(b->s0, b->join_ev[j], 0));
    }
    ck(cudaMemcpyAsync(b->h_report, b->d_report, n * sizeof(hyb::DevState), cudaMemcpyDeviceToHost, b->s0));
    return e;
}

struct SavedState {
    std::vector<cudaStream_t> stream;
    std::vector<int> cur;
    std::vector<void*> phi, old;
};

SavedState enter(hyb_batch* b, int q) {
    SavedState sv;
    for (size_t i = 0; i < b->probs.size(); ++i) {
        hyb_problem* p = b->probs[i];
        sv.stream.push_back(p->stream); sv.cur.push_back(p->cur); sv.phi.push_back(p->sn_phi); sv.old.push_back(p->sn_phi_old);
        p->cur = b->cur0[i] ^ q;
    }
    return sv;
}

void leave(hyb_batch* b, const SavedState& sv) {
    for (size_t i = 0; i < b->probs.size(); ++i) {
        hyb_problem* p = b->probs[i];
        p->stream = sv.stream[i]; p->cur = sv.cur[i]; p->sn_phi = sv.phi[i]; p->sn_phi_old = sv.old[i];
    }
}

void record_mid(hyb_batch* b, int q) {
    const size_t n = b->probs.size();
    b->phi_mid[q].assign(n, nullptr);
    b->old_mid[q].assign(n, nullptr);
    for (size_t i = 0; i < n; ++i) { b->phi_mid[q][i] = b->probs[i]->sn_phi; b->old_mid[q][i] = b->probs[i]->sn_phi_old; }
}

// Record one batch step of parity q as two graphs (phases 0 and 1).
hyb_status capture(hyb_batch* b, int q) {
    const SavedState sv = enter(b, q);
    cudaError_t e = cudaSuccess;
    for (int phase = 0; phase < 2 && e == cudaSuccess; ++phase) {
        e = cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t ei = issue_phase(b, q, phase);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->s0, &g);
        e = ei != cudaSuccess ? ei : e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[q][phase], g, 0);
        if (g) cudaGraphDestroy(g);
        if (phase == 0) record_mid(b, q);
    }
    leave(b, sv);
    if (e != cudaSuccess) {
        drop_graphs(b);
        return bfail(b, HYB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    return HYB_OK;
}

// Continue the source iteration of problem i (phase-0 cap reached) until its device flag is set,
// with an even number of further iterations so phase 1 finds the newest iterate where it was
// recorded (an iteration after convergence only carries the solution forward).
hyb_status finish_iterations(hyb_batch* b, int q, size_t i) {
    hyb_problem* p = b->probs[i];
    void* ph = p->sn_phi; void* po = p->sn_phi_old; cudaStream_t ps = p->stream;
    p->sn_phi = b->phi_mid[q][i]; p->sn_phi_old = b->old_mid[q][i];
    p->stream = b->s0;
    hyb_status rc = HYB_OK;
    int extra = 0;
    for (int k = b->kmax[i]; k < p->d.sn_max_iter; ++k) {
        if (hyb::sn_iteration(p, 0) != cudaSuccess) { rc = HYB_ECUDA; break; }
        ++extra;
        if (extra % 2 == 0) {
            cudaMemcpyAsync(&p->st_host->sn_conv, &p->st->sn_conv, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->s0);
            if (cudaStreamSynchronize(b->s0) != cudaSuccess) { rc = HYB_ECUDA; break; }
            if (p->st_host->sn_conv) break;
        }
    }
    if (extra % 2 == 1 && rc == HYB_OK && hyb::sn_iteration(p, 0) != cudaSuccess) rc = HYB_ECUDA;
    cudaStreamSynchronize(b->s0);
    p->sn_phi = ph; p->sn_phi_old = po; p->stream = ps;
    return rc == HYB_OK ? HYB_OK : bfail(b, rc, "eager source iteration");
}

// Takes the batch's problem set: per-problem device buffers grow only, so replacing the set
// (continuous batching) allocates nothing once the largest set has been seen.
hyb_status load_problems(hyb_batch* b, hyb_problem* const* problems, int32_t n) {
    const int prec = problems[0] ? problems[0]->prec : 0;
    std::vector<hyb_problem*> probs;
    for (int i = 0; i < n; ++i) {
        hyb_problem* p = problems[i];
        if (!p || p->prec != prec) return bfail(b, HYB_EINVAL, "problems must share one precision");
        if (p->leg_done) return bfail(b, HYB_ESTATE, "problems must be at a step boundary");
        if (p->d.n_s == HYB_NS_INF) return bfail(b, HYB_EINVAL, "N_s = infinity problems are stepped alone");
        if (p->d.sampler == HYB_HALTON) return bfail(b, HYB_EINVAL, "Halton problems are stepped alone");
        if (p->d.remap_variant != 0) return bfail(b, HYB_EINVAL, "the additive remap variant is stepped alone");
        // a step graph replays one sort decision: a census sorted on some steps only is stepped alone
        if (p->d.census_order >= 1 && p->d.sort_every > 1)
            return bfail(b, HYB_EINVAL, "a census sort interval (sort_every > 1) is stepped alone");
        if (p->d.leg_sort_every > 0) return bfail(b, HYB_EINVAL, "the phased leg (leg_sort_every > 0) is stepped alone");
        probs.push_back(p);
    }
    if (!b->probs.empty() && prec != b->prec) return bfail(b, HYB_EINVAL, "a batch keeps one precision");
    b->prec = prec;
    b->probs = probs;
    b->cur0.clear(); b->kmax.clear();
    b->ntab_max = 0;
    for (hyb_problem* p : probs) {
        b->cur0.push_back(p->cur);
        b->kmax.push_back(std::max(8, p->last_sn_iters + 3));
        b->ntab_max = std::max(b->ntab_max, hyb::leg_ntab(p));
    }
    b->parity = 0;
    const size_t ab = hyb::leg_args_bytes(b->prec);
    if ((size_t)n > b->cap_probs) {
        const size_t cap = std::max<size_t>((size_t)n, 2 * b->cap_probs);
        for (int q = 0; q < 2; ++q) { if (b->d_args[q]) cudaFree(b->d_args[q]); b->d_args[q] = nullptr; }
        if (b->d_report) cudaFree(b->d_report);
        if (b->h_report) cudaFreeHost(b->h_report);
        b->d_report = nullptr; b->h_report = nullptr;
        b->cap_probs = 0;
        for (int q = 0; q < 2; ++q)
            if (cudaMalloc(&b->d_args[q], ab * cap) != cudaSuccess) return bfail(b, HYB_ENOMEM, "args");
        if (cudaMalloc(&b->d_report, cap * sizeof(hyb::DevState)) != cudaSuccess ||
            cudaMallocHost(&b->h_report, cap * sizeof(hyb::DevState)) != cudaSuccess)
            return bfail(b, HYB_ENOMEM, "report");
        b->cap_probs = cap;
    }
    std::vector<unsigned char> host(ab * n);
    for (int q = 0; q < 2; ++q) {
        for (int i = 0; i < n; ++i) hyb::leg_args_host(b->probs[i], b->cur0[i] ^ q, host.data() + ab * i);
        if (cudaMemcpy(b->d_args[q], host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, HYB_ECUDA, "args upload");
    }
    // programmatic dependent launch is kept for problems stepped alone: in the batch's multi-stream
    // step graphs it measured slower (256 problems: 73 -> 101 ms per step). Members launch normally
    // once the batch holds them (problems that left the set may already be destroyed: they get it
    // back when they are next stepped alone)
    for (hyb_problem* p : probs) {
        // a bank pre-pass left pending by a failed single-problem step is ordered and forgotten:
        // the batch re-streams every slot itself
        if (hyb::drop_bank_prepass(p) != cudaSuccess) return bfail(b, HYB_ECUDA, "bank pre-pass");
    }
    // nothing below can fail: the members' state changes only for a batch that holds them
    for (hyb_problem* p : probs) {
        p->pdl = false;
        p->births_step = -1;   // the batch draws its members' births into their buffers itself
    }
    return HYB_OK;
}

}  // namespace

extern "C" {

HYB_API hyb_status hyb_batch_create(hyb_problem* const* problems, int32_t n, void* cuda_stream, hyb_batch** out) {
    if (!problems || n < 1 || !out) return bfail(nullptr, HYB_EINVAL, "need at least one problem");
    *out = nullptr;
    hyb_batch* b = new (std::nothrow) hyb_batch();
    if (!b) return bfail(nullptr, HYB_ENOMEM, "host allocation");
    b->prec = problems[0] ? problems[0]->prec : 0;
    b->s0 = (cudaStream_t)cuda_stream;
    if (!b->s0) {   // graphs cannot be recorded on the legacy default stream
        if (cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return bfail(nullptr, HYB_ECUDA, "stream");
        }
        b->own_s0 = true;
    }
    auto fail_all = [&](hyb_status s, std::string m) {   // m by value: it may be b->err
        hyb_batch_destroy(b);
        g_batch_err = std::move(m);
        return s;
    };
    if (cudaMalloc(&b->d_head, 2 * sizeof(int)) != cudaSuccess) return fail_all(HYB_ENOMEM, "queue heads");
    if (cudaMalloc(&b->d_V, HYB_SOBOL_DIMS * 32 * 4) != cudaSuccess) return fail_all(HYB_ENOMEM, "table");
    if (cudaMemcpy(b->d_V, hyb::sobol_table_host(), HYB_SOBOL_DIMS * 32 * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail_all(HYB_ECUDA, "table upload");
    if (cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
        cudaEventCreate(&b->evl0) != cudaSuccess || cudaEventCreate(&b->evl1) != cudaSuccess)
        return fail_all(HYB_ECUDA, "events");
    hyb_status s = load_problems(b, problems, n);
    if (s == HYB_OK) s = hyb_batch_set_tuning(b, &b->tune);
    if (s != HYB_OK) return fail_all(s, b->err);
    *out = b;
    return HYB_OK;
}

HYB_API hyb_status hyb_batch_set_problems(hyb_batch* b, hyb_problem* const* problems, int32_t n) {
    if (!b || !problems || n < 1) return bfail(b, HYB_EINVAL, "need at least one problem");
    if (b->s0 && cudaStreamSynchronize(b->s0) != cudaSuccess) return bfail(b, HYB_ECUDA, "stream");
    drop_graphs(b);
    hyb_status s = load_problems(b, problems, n);
    if (s != HYB_OK) return s;
    return build_chunks(b);
}

HYB_API hyb_status hyb_batch_set_tuning(hyb_batch* b, const hyb_batch_tuning* t) {
    if (!b || !t) return bfail(b, HYB_EINVAL, "null argument");
    if ((t->block != 128 && t->block != 256) || t->chunk < 32 || t->ctas_per_sm < 0 || t->ctas_per_sm > 16 ||
        t->streams < 1 || t->streams > 64 || (t->use_graph != 0 && t->use_graph != 1))
        return bfail(b, HYB_EINVAL, "tuning out of range (block 128|256, chunk >= 32, streams 1..64, use_graph 0|1)");
    b->tune = *t;
    drop_graphs(b);
    for (auto s : b->pool) cudaStreamDestroy(s);
    for (auto e : b->join_ev) cudaEventDestroy(e);
    b->pool.clear(); b->join_ev.clear();
    for (int j = 0; j < t->streams; ++j) {
        cudaStream_t s; cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bfail(b, HYB_ECUDA, "stream");
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bfail(b, HYB_ECUDA, "event");
        b->pool.push_back(s); b->join_ev.push_back(e);
    }
    return build_chunks(b);
}

HYB_API hyb_status hyb_batch_step(hyb_batch* b, int32_t nsteps, hyb_leg_stats* per_problem) {
    if (!b || nsteps < 0) return bfail(b, HYB_EINVAL, "bad arguments");
    const size_t n = b->probs.size();
    for (int32_t it = 0; it < nsteps; ++it) {
        const int q = b->parity;
        const bool graph = b->tune.use_graph != 0;
        SavedState sv;
        if (graph && (!b->exec[q][0] || !b->exec[q][1])) {
            hyb_status s = capture(b, q);
            if (s != HYB_OK) return s;
        }
        if (cudaEventRecord(b->ev0, b->s0) != cudaSuccess) return bfail(b, HYB_ECUDA, "event");
        if (graph) {
            if (cudaGraphLaunch(b->exec[q][0], b->s0) != cudaSuccess || cudaStreamSynchronize(b->s0) != cudaSuccess)
                return bfail(b, HYB_ECUDA, "graph launch (leg and source iteration)");
        } else {
            sv = enter(b, q);
            const cudaError_t e = issue_phase(b, q, 0);
            record_mid(b, q);
            leave(b, sv);
            if (e != cudaSuccess || cudaStreamSynchronize(b->s0) != cudaSuccess)
                return bfail(b, HYB_ECUDA, "eager phase 0");
        }
        bool recapture = false;
        for (size_t i = 0; i < n; ++i) {
            if (b->h_report[i].sn_conv) continue;
            hyb_status s = finish_iterations(b, q, i);
            if (s != HYB_OK) return s;
            b->kmax[i] = std::min(b->probs[i]->d.sn_max_iter, std::max(2 * b->kmax[i], b->probs[i]->st_host->sn_iters + 2));
            recapture = true;
        }
        if (graph) {
            if (cudaGraphLaunch(b->exec[q][1], b->s0) != cudaSuccess) return bfail(b, HYB_ECUDA, "graph launch (remap)");
        } else {
            sv = enter(b, q);
            for (size_t i = 0; i < n; ++i) { b->probs[i]->sn_phi = b->phi_mid[q][i]; b->probs[i]->sn_phi_old = b->old_mid[q][i]; }
            const cudaError_t e = issue_phase(b, q, 1);
            leave(b, sv);
            if (e != cudaSuccess) return bfail(b, HYB_ECUDA, "eager phase 1");
        }
        if (cudaEventRecord(b->ev1, b->s0) != cudaSuccess || cudaStreamSynchronize(b->s0) != cudaSuccess)
            return bfail(b, HYB_ECUDA, "step completion");
        b->parity ^= 1;
        hyb_status bad = HYB_OK;
        for (size_t i = 0; i < n; ++i) {
            hyb_problem* p = b->probs[i];
            const hyb::DevState& r = b->h_report[i];
            p->cur ^= 1;
            p->step += 1;
            p->last_sn_iters = r.sn_iters;
            p->sn_warm = p->d.sn_warm_start != 0;
            p->leg_done = p->sn_done = false;
            if (r.status & hyb::kStBounds) bad = HYB_EBOUNDS;
            else if ((r.status & hyb::kStSegments) && bad == HYB_OK) bad = HYB_ETIMEOUT;
        }
        if (recapture && graph) drop_graphs(b);
        if (bad != HYB_OK) return bfail(b, bad, "a problem of the batch reported a device check failure");
    }
    if (per_problem) {
        float ms = 0, ms_leg = 0;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        cudaEventElapsedTime(&ms_leg, b->evl0, b->evl1);
        for (size_t i = 0; i < n; ++i) {
            hyb_problem* p = b->probs[i];
            const hyb::DevState& h = b->h_report[i];
            hyb_leg_stats& s = per_problem[i];
            std::memset(&s, 0, sizeof(s));
            s.histories = (int64_t)h.histories; s.segments = (int64_t)h.segments; s.collisions = (int64_t)h.collisions;
            s.leaked = (int64_t)h.leaked; s.census = (int64_t)h.census; s.killed = (int64_t)h.killed;
            s.reached_limit = (int64_t)h.reached; s.errors = (int64_t)h.errors; s.tally_adds = (int64_t)h.tally_adds;
            const double iw = std::ldexp(1.0, -h.k_w);
            s.w_source = hyb::acc128_to_double(h.w_source.lo, h.w_source.hi, iw);
            s.w_absorbed = hyb::acc128_to_double(h.w_absorbed.lo, h.w_absorbed.hi, iw);
            s.w_leaked = hyb::acc128_to_double(h.w_leaked.lo, h.w_leaked.hi, iw);
            s.w_census = hyb::acc128_to_double(h.w_census.lo, h.w_census.hi, iw);
            s.w_handoff = hyb::acc128_to_double(h.w_handoff.lo, h.w_handoff.hi, iw);
            s.w_killed = hyb::acc128_to_double(h.w_killed.lo, h.w_killed.hi, iw);
            s.sn_iterations = h.sn_iters;
            s.combed = h.comb_on;
            s.bank_size = h.n_bank;
            s.ms = ms;
            s.ms_leg = ms_leg;
            (void)p;
        }
    }
    return HYB_OK;
}

HYB_API hyb_status hyb_batch_destroy(hyb_batch* b) {
    if (!b) return HYB_OK;
    if (b->s0) cudaStreamSynchronize(b->s0); else cudaDeviceSynchronize();
    drop_graphs(b);
    for (auto s : b->pool) cudaStreamDestroy(s);
    for (auto e : b->join_ev) cudaEventDestroy(e);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->evl0) cudaEventDestroy(b->evl0);
    if (b->evl1) cudaEventDestroy(b->evl1);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    for (int q = 0; q < 2; ++q) if (b->d_args[q]) cudaFree(b->d_args[q]);
    if (b->d_chunks) cudaFree(b->d_chunks);
    if (b->d_head) cudaFree(b->d_head);
    if (b->d_bchunks) cudaFree(b->d_bchunks);
    if (b->d_report) cudaFree(b->d_report);
    if (b->h_report) cudaFreeHost(b->h_report);
    if (b->d_V) cudaFree(b->d_V);
    if (b->own_s0 && b->s0) cudaStreamDestroy(b->s0);
    delete b;
    return HYB_OK;
}

HYB_API const char* hyb_batch_last_error(const hyb_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
