// Batched stepping of independent filter instances (contexts). Every phase of
// a step runs over the blocks of all instances at once: grouped launches
// (k_group<Op>: a block map names the instance and block each CTA runs, a
// table holds each instance's arguments), and for the two phases made of
// dependent sub-steps, the LSH/sort phase and the posterior, one cooperative
// persistent launch each with grid barriers between the sub-steps. A batch
// step is about a dozen launches whatever the number of instances, all on the
// batch's stream. The launches are captured
// once into a CUDA graph per pinned staging slot and every batch step replays
// one; the host fills the other slot (scans, odometry, LSH draw, step
// counter) while a step runs. Before the capture, the likelihood's scan split
// of each instance is picked by timing: alone first, then as a policy over the
// instances' grouped launch.
#include "mp_internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

// ---------------------------------------------------------------------------
// mp_group: device tables of the planners
// ---------------------------------------------------------------------------
const void* mp_group::upload(const void* host, size_t bytes) {
    if (err) return nullptr;
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        err = e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA;
        return nullptr;
    }
    arena.push_back(d);
    if (bytes && cudaMemcpy(d, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        err = MP_ECUDA;
        return nullptr;
    }
    return d;
}

void* mp_group::scratch(size_t bytes) {
    if (err) return nullptr;
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        err = e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA;
        return nullptr;
    }
    arena.push_back(d);
    if (cudaMemset(d, 0, bytes ? bytes : 1) != cudaSuccess) {
        err = MP_ECUDA;
        return nullptr;
    }
    return d;
}

const GBlk* mp_group::block_map(const std::vector<int64_t>& blocks, unsigned* nblk, const std::vector<int>& which,
                                const std::vector<int>& ysplit) {
    std::vector<GBlk> m;
    auto add = [&](int i) {
        const int ny = ysplit.empty() ? 1 : ysplit[i];
        for (int64_t b = 0; b < blocks[i]; ++b)
            for (int y = 0; y < ny; ++y) m.push_back(GBlk{i, (int32_t)b, y, 0});
    };
    if (which.empty())
        for (int i = 0; i < size(); ++i) add(i);
    else
        for (int i : which) add(i);
    *nblk = (unsigned)m.size();
    if (m.empty()) return nullptr;
    return upload(m);
}

void mp_group::release() {
    for (void* p : arena) cudaFree(p);
    arena.clear();
    if (scan_dev) cudaFree(scan_dev);
    if (sd_dev) cudaFree(sd_dev);
    scan_dev = nullptr;
    sd_dev = nullptr;
}

struct mp_batch {
    mp_group G;
    int n = 0;
    std::vector<int> nbr_cur0;       // each instance's current neighbour list when the graphs were captured
    int64_t scan_floats = 0;         // floats of one staging slot
    cudaStream_t origin = nullptr;
    StepDev* stage = nullptr;        // pinned, [2][n]
    float* scans = nullptr;          // pinned, [2][scan_floats]
    std::vector<cudaEvent_t> join;   // per instance: work queued on its own stream before a step
    cudaEvent_t done[2] = {nullptr, nullptr};
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int64_t steps = 0;
};

namespace {

void batch_free(mp_batch* b) {
    if (!b) return;
    if (b->origin) cudaStreamSynchronize(b->origin);
    for (int p = 0; p < 2; ++p) {
        if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
        if (b->graph[p]) cudaGraphDestroy(b->graph[p]);
        if (b->done[p]) cudaEventDestroy(b->done[p]);
    }
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->stage) cudaFreeHost(b->stage);
    if (b->scans) cudaFreeHost(b->scans);
    b->G.release();
    delete b;
}

int batch_err(cudaError_t e, const char* what) {
    return mp_fail_noctx(e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA, "mp_batch: %s: %s", what,
                         cudaGetErrorString(e));
}

#define B_CUDA(x)                                        \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return batch_err(e_, #x); \
    } while (0)

// Issues the operations of a plan on stream s (directly, or into a capture).
int run_plan(const std::vector<GOp>& plan, cudaStream_t s) {
    for (const GOp& o : plan) {
        if (o.kind == GOp::KERNEL) {
            void* args[2] = {(void*)&o.tab, (void*)&o.map};
            B_CUDA(cudaLaunchKernel(o.func, dim3(o.grid), dim3(o.block), args, 0, s));
        } else if (o.kind == GOp::COOP) {
            B_CUDA(launch_coop(o.func, o.grid, o.block, (void*)o.arg, s));
        } else if (o.kind == GOp::MEMSET) {
            B_CUDA(cudaMemsetAsync(o.dst, 0, o.bytes, s));
        } else {
            B_CUDA(cudaMemcpyAsync(o.dst, o.src, o.bytes, cudaMemcpyDeviceToDevice, s));
        }
    }
    return MP_OK;
}

// Every stage of one step, for neighbour-list parity p.
int plan_step(mp_group* G, int p, std::vector<GOp>& plan) {
    int rc;
    if ((rc = mp_plan_predict(G, p, plan))) return rc;
    if ((rc = mp_plan_scan(G, p, plan))) return rc;
    if ((rc = mp_plan_lsh_sort(G, p, plan))) return rc;
    if ((rc = mp_plan_merge(G, p, plan))) return rc;
    if ((rc = mp_plan_likelihood(G, p, plan))) return rc;
    if ((rc = mp_plan_solve_svgd(G, p, plan))) return rc;
    return mp_plan_posterior(G, p, plan);
}

// Time the likelihood of c (its current particles and scan) for each split
// and keep the fastest. The scan, LSH and sort stages run first so that the
// particle order the kernel reads is set.
int autotune_split(mp_ctx* c) {
    int rc;
    if ((rc = mp_run_stages(c, MP_STAGE_SCAN | MP_STAGE_LSH | MP_STAGE_SORT))) return rc;
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    const int chunks = (c->n_scan + 255) / 256;
    float best_ms = 1e30f;
    int best = 1;
    for (int split = 1; split <= 16; split *= 2) {
        if (split > 1 && split > chunks) break;
        c->lk_split = split;
        if ((rc = mp_run_stages(c, MP_STAGE_LIKELIHOOD))) break;   // warm-up
        B_CUDA(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < 3; ++r)
            if ((rc = mp_run_stages(c, MP_STAGE_LIKELIHOOD))) break;
        B_CUDA(cudaEventRecord(e1, c->stream));
        B_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        B_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = split; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->lk_split = best;
    return rc;
}

// The grouped likelihood of all instances with their current splits, timed
// on the batch stream (3 launches after one warm-up).
int time_group_likelihood(mp_batch* b, float* ms_out) {
    mp_group T;   // a scratch group for this policy's tables
    T.ctx = b->G.ctx;
    T.n_scan = b->G.n_scan;
    T.scan_off = b->G.scan_off;
    std::vector<GOp> plan;
    int rc = mp_plan_likelihood(&T, 0, plan);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == MP_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = MP_ECUDA;
    if (rc == MP_OK) rc = run_plan(plan, b->origin);
    if (rc == MP_OK && cudaEventRecord(e0, b->origin) != cudaSuccess) rc = MP_ECUDA;
    for (int r = 0; r < 3 && rc == MP_OK; ++r) rc = run_plan(plan, b->origin);
    if (rc == MP_OK && cudaEventRecord(e1, b->origin) != cudaSuccess) rc = MP_ECUDA;
    if (rc == MP_OK) {
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) rc = batch_err(e, "cudaEventSynchronize(e1)");
        else if (cudaEventElapsedTime(ms_out, e0, e1) != cudaSuccess) rc = MP_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(b->origin);
    T.scan_dev = nullptr;
    T.sd_dev = nullptr;
    T.release();
    return rc;
}

}  // namespace

extern "C" {

int mp_batch_create(mp_batch** out, mp_ctx* const* ctxs, int n, const int32_t* n_scan,
                    const float* const* tune_scans, void* cuda_stream) {
    if (!out || !ctxs || n < 1 || !n_scan || !cuda_stream)
        return mp_fail_noctx(MP_EINVAL, "mp_batch_create: NULL argument or no instance");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        mp_ctx* c = ctxs[i];
        if (!c || c->n == 0 || c->timing || n_scan[i] < 1 || n_scan[i] > c->p.max_scan)
            return mp_fail_noctx(MP_EINVAL, "mp_batch_create: instance %d: uninitialised, timed, or a scan size "
                                            "outside [1, max_scan]", i);
        if (c->precision != MP_PREC_FP32)
            return mp_fail_noctx(MP_EINVAL, "mp_batch_create: instance %d: batched instances use the FP32 "
                                            "likelihood", i);
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == c)
                return mp_fail_noctx(MP_EINVAL, "mp_batch_create: instances %d and %d are the same context", k, i);
    }
    mp_batch* b = new mp_batch();
    b->n = n;
    b->origin = (cudaStream_t)cuda_stream;
    b->G.ctx.assign(ctxs, ctxs + n);
    b->G.n_scan.assign(n_scan, n_scan + n);
    b->G.scan_off.resize(n);
    b->join.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        b->G.scan_off[i] = b->scan_floats;
        b->scan_floats += 3 * (int64_t)n_scan[i];
    }
    int rc = MP_OK;
    auto fail = [&](int code) {
        batch_free(b);
        return code;
    };
    cudaError_t e = cudaHostAlloc((void**)&b->stage, 2 * sizeof(StepDev) * n, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->scans, 2 * sizeof(float) * b->scan_floats, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->G.scan_dev, sizeof(float) * b->scan_floats);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->G.sd_dev, sizeof(StepDev) * n);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = cudaEventCreateWithFlags(&b->done[p], cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(batch_err(e, "allocation"));
    memset(b->stage, 0, 2 * sizeof(StepDev) * n);
    memset(b->scans, 0, 2 * sizeof(float) * b->scan_floats);

    // tile choice: each instance's split timed alone, then three policies
    // timed as the grouped launch of all instances (alone, a split helps a
    // small instance fill the GPU; together, the other instances fill it and
    // the split's atomics may not pay): the splits timed alone, none, and the
    // timed splits only for instances with less than 3 waves of particle blocks
    std::vector<int> alone(n, 1);
    bool tuned = tune_scans != nullptr;
    for (int i = 0; i < n; ++i) {
        mp_ctx* c = b->G.ctx[i];
        c->lk_split = 1;
        if (tune_scans && tune_scans[i]) {
            if ((rc = mp_set_scan(c, tune_scans[i], n_scan[i]))) return fail(rc);
            if ((rc = autotune_split(c))) return fail(rc);
            alone[i] = c->lk_split;
        } else {
            tuned = false;
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(MP_ECUDA);
    }
    if (tuned && n > 1) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        auto policy = [&](int pol, int i) {
            const int64_t blocks = (b->G.ctx[i]->n + 255) / 256;
            return pol == 0 ? alone[i] : pol == 1 ? 1 : (blocks < 3 * (int64_t)sms ? alone[i] : 1);
        };
        float best_ms = 1e30f;
        int best = 0;
        for (int pol = 0; pol < 3; ++pol) {
            for (int i = 0; i < n; ++i) b->G.ctx[i]->lk_split = policy(pol, i);
            float ms = 0.f;
            if ((rc = time_group_likelihood(b, &ms))) return fail(rc);
            if (ms < best_ms) { best_ms = ms; best = pol; }
        }
        for (int i = 0; i < n; ++i) b->G.ctx[i]->lk_split = policy(best, i);
    }

    // one graph per staging slot: the step inputs copied in, then every
    // stage as one grouped launch. The merge swaps the two neighbour-list
    // buffers (a host-side index): graph p reads list nbr_cur0 ^ p, so replays
    // alternate slots and the host index is swapped after each replay
    b->nbr_cur0.resize(n);
    for (int i = 0; i < n; ++i) b->nbr_cur0[i] = b->G.ctx[i]->nbr_cur;
    for (int p = 0; p < 2; ++p) {
        std::vector<GOp> plan;
        if ((rc = plan_step(&b->G, p, plan))) return fail(rc);
        e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(batch_err(e, "begin capture"));
        cudaMemcpyAsync(b->G.scan_dev, b->scans + p * b->scan_floats, sizeof(float) * b->scan_floats,
                        cudaMemcpyHostToDevice, b->origin);
        cudaMemcpyAsync(b->G.sd_dev, b->stage + p * n, sizeof(StepDev) * n, cudaMemcpyHostToDevice, b->origin);
        rc = run_plan(plan, b->origin);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->origin, &g);
        if (rc != MP_OK) {
            if (g) cudaGraphDestroy(g);
            return fail(rc);
        }
        if (e != cudaSuccess) return fail(batch_err(e, "end capture"));
        b->graph[p] = g;
        e = cudaGraphInstantiate(&b->exec[p], g, 0);
        if (e != cudaSuccess) return fail(batch_err(e, "instantiate"));
    }
    *out = b;
    return MP_OK;
}

int mp_batch_step(mp_batch* b, const float* const* scans, const double* odom_T, const double* odom_cov) {
    if (!b || !scans) return mp_fail_noctx(MP_EINVAL, "mp_batch_step: NULL batch or scans");
    const int p = (int)(b->steps & 1);
    B_CUDA(cudaEventSynchronize(b->done[p]));   // the launch that last read slot p
    int rc;
    for (int i = 0; i < b->n; ++i) {
        mp_ctx* c = b->G.ctx[i];
        if (!scans[i]) return mp_fail_noctx(MP_EINVAL, "mp_batch_step: NULL scan of instance %d", i);
        if (c->nbr_cur != (b->nbr_cur0[i] ^ p))
            return mp_fail_noctx(MP_EINVAL, "mp_batch_step: instance %d was stepped outside the batch", i);
        memcpy(b->scans + p * b->scan_floats + b->G.scan_off[i], scans[i], sizeof(float) * 3 * (size_t)b->G.n_scan[i]);
        if ((rc = mp_set_odometry(c, odom_T ? odom_T + 16 * i : nullptr, odom_cov ? odom_cov + 36 * i : nullptr)))
            return rc;
        draw_lsh(c);
        fill_step_host(c, b->stage + p * b->n + i);
        // work queued on an instance's own stream before this step comes first
        B_CUDA(cudaEventRecord(b->join[i], c->stream));
        B_CUDA(cudaStreamWaitEvent(b->origin, b->join[i], 0));
    }
    B_CUDA(cudaGraphLaunch(b->exec[p], b->origin));
    B_CUDA(cudaEventRecord(b->done[p], b->origin));
    for (int i = 0; i < b->n; ++i) {
        mp_ctx* c = b->G.ctx[i];
        // later calls on the instance (mp_get_posterior, mp_step) wait for the graph
        B_CUDA(cudaStreamWaitEvent(c->stream, b->done[p], 0));
        c->n_scan = b->G.n_scan[i];
        c->nbr_cur ^= 1;
        c->step++;
    }
    b->steps++;
    return MP_OK;
}

int mp_batch_split(mp_batch* b, int i, int* split) {
    if (!b || !split || i < 0 || i >= b->n) return mp_fail_noctx(MP_EINVAL, "mp_batch_split: invalid argument");
    *split = b->G.ctx[i]->lk_split > 1 ? b->G.ctx[i]->lk_split : 1;
    return MP_OK;
}

int mp_stream_create(void** stream) {
    if (!stream) return mp_fail_noctx(MP_EINVAL, "mp_stream_create: invalid argument");
    cudaStream_t s = nullptr;
    B_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    *stream = (void*)s;
    return MP_OK;
}

int mp_stream_destroy(void* stream) {
    if (!stream) return mp_fail_noctx(MP_EINVAL, "mp_stream_destroy: invalid argument");
    B_CUDA(cudaStreamDestroy((cudaStream_t)stream));
    return MP_OK;
}

int mp_batch_destroy(mp_batch* b) {
    if (!b) return mp_fail_noctx(MP_EINVAL, "mp_batch_destroy: invalid argument");
    batch_free(b);
    return MP_OK;
}

}  // extern "C"
