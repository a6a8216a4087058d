// Batched stepping of independent filter instances (contexts): one step of
// every instance is captured once into a CUDA graph, each instance on its own
// stream branch (forked from and joined into an origin stream), and every
// batch step replays it. The values a step takes from the host (the scan, the
// odometry, the LSH draw, the step counter) are copied by the graph from
// pinned staging slots that the host fills before the launch; two slots (two
// graphs) let the host prepare step s + 1 while step s runs. Before the
// capture, the likelihood's scan split of each instance is picked by timing:
// alone first, then as a policy across the instances running together.
#include "mp_internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

struct mp_batch {
    int n = 0;
    std::vector<mp_ctx*> ctx;
    std::vector<int32_t> n_scan;
    std::vector<int> nbr_cur0;       // each instance's current neighbour list when the graphs were captured
    std::vector<int64_t> scan_off;   // offset of instance i's scan in a slot (floats)
    int64_t scan_floats = 0;         // floats of one slot
    cudaStream_t origin = nullptr;
    StepDev* stage = nullptr;        // pinned, [2][n]
    float* scans = nullptr;          // pinned, [2][scan_floats]
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;   // per instance
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
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->stage) cudaFreeHost(b->stage);
    if (b->scans) cudaFreeHost(b->scans);
    for (mp_ctx* c : b->ctx) c->batch_slot = nullptr;
    delete b;
}

int batch_err(cudaError_t e, const char* what) {
    fprintf(stderr, "mp_batch: %s: %s\n", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA;
}

#define B_CUDA(x)                                        \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return batch_err(e_, #x); \
    } while (0)

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

// All instances' likelihood stages launched together (each on its own stream,
// forked from and joined into origin), timed on origin: the stage only writes
// per-step outputs, so the instances' state is untouched.
int time_concurrent_likelihood(mp_batch* b, float* ms_out) {
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    int rc = MP_OK;
    B_CUDA(cudaEventRecord(e0, b->origin));
    for (int rep = 0; rep < 3 && rc == MP_OK; ++rep) {
        B_CUDA(cudaEventRecord(b->fork, b->origin));
        for (int i = 0; i < b->n && rc == MP_OK; ++i) {
            mp_ctx* c = b->ctx[i];
            B_CUDA(cudaStreamWaitEvent(c->stream, b->fork, 0));
            rc = mp_run_stages(c, MP_STAGE_LIKELIHOOD);
            B_CUDA(cudaEventRecord(b->join[i], c->stream));
            B_CUDA(cudaStreamWaitEvent(b->origin, b->join[i], 0));
        }
    }
    B_CUDA(cudaEventRecord(e1, b->origin));
    B_CUDA(cudaEventSynchronize(e1));
    B_CUDA(cudaEventElapsedTime(ms_out, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" {

int mp_batch_create(mp_batch** out, mp_ctx* const* ctxs, int n, const int32_t* n_scan,
                    const float* const* tune_scans, void* cuda_stream) {
    if (!out || !ctxs || n < 1 || !n_scan || !cuda_stream) return MP_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        mp_ctx* c = ctxs[i];
        if (!c || c->n == 0 || !c->stream || c->timing || n_scan[i] < 1 || n_scan[i] > c->p.max_scan) {
            fprintf(stderr, "mp_batch_create: instance %d: uninitialised, on the default stream, timed, or a scan "
                            "size outside [1, max_scan]\n", i);
            return MP_EINVAL;
        }
        if (c->stream == (cudaStream_t)cuda_stream) {
            fprintf(stderr, "mp_batch_create: instance %d uses the batch's own stream\n", i);
            return MP_EINVAL;
        }
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == c || ctxs[k]->stream == c->stream) {
                fprintf(stderr, "mp_batch_create: instances %d and %d share a context or a stream\n", k, i);
                return MP_EINVAL;
            }
    }
    mp_batch* b = new mp_batch();
    b->n = n;
    b->ctx.assign(ctxs, ctxs + n);
    b->n_scan.assign(n_scan, n_scan + n);
    b->origin = (cudaStream_t)cuda_stream;
    b->join.assign(n, nullptr);
    b->scan_off.resize(n);
    for (int i = 0; i < n; ++i) {
        b->scan_off[i] = b->scan_floats;
        b->scan_floats += 3 * (int64_t)n_scan[i];
    }
    int rc = MP_OK;
    auto fail = [&](int code) {
        batch_free(b);
        return code;
    };
    cudaError_t e = cudaHostAlloc((void**)&b->stage, 2 * sizeof(StepDev) * n, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->scans, 2 * sizeof(float) * b->scan_floats, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = cudaEventCreateWithFlags(&b->done[p], cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(batch_err(e, "allocation"));
    memset(b->stage, 0, 2 * sizeof(StepDev) * n);
    memset(b->scans, 0, 2 * sizeof(float) * b->scan_floats);

    // tile choice: each instance's split timed alone, then three policies
    // timed with all instances running together (alone, a split helps a small
    // instance fill the GPU; together, the others fill it and the split's
    // atomics may not pay): the splits timed alone, none, and the timed splits
    // only for instances with less than one wave of particle blocks
    std::vector<int> alone(n, 1);
    bool tuned = tune_scans != nullptr;
    for (int i = 0; i < n; ++i) {
        mp_ctx* c = b->ctx[i];
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
        float best_ms = 1e30f;
        int best = 0;
        for (int pol = 0; pol < 3; ++pol) {
            for (int i = 0; i < n; ++i) {
                const int64_t blocks = (b->ctx[i]->n + 255) / 256;
                b->ctx[i]->lk_split = pol == 0 ? alone[i] : pol == 1 ? 1 : (blocks < 3 * (int64_t)sms ? alone[i] : 1);
            }
            float ms = 0.f;
            if ((rc = time_concurrent_likelihood(b, &ms))) return fail(rc);
            if (ms < best_ms) { best_ms = ms; best = pol; }
        }
        for (int i = 0; i < n; ++i) {
            const int64_t blocks = (b->ctx[i]->n + 255) / 256;
            b->ctx[i]->lk_split = best == 0 ? alone[i] : best == 1 ? 1 : (blocks < 3 * (int64_t)sms ? alone[i] : 1);
        }
    }

    // one graph per staging slot: every instance's full step on its own branch.
    // The merge stage swaps the two neighbour-list buffers (host-side index):
    // graph 0 reads the current one, graph 1 the other, so replays alternate
    // slots and the host index is swapped after each replay
    b->nbr_cur0.resize(n);
    for (int i = 0; i < n; ++i) b->nbr_cur0[i] = b->ctx[i]->nbr_cur;
    for (int p = 0; p < 2; ++p) {
        e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(batch_err(e, "begin capture"));
        cudaEventRecord(b->fork, b->origin);
        for (int i = 0; i < n && rc == MP_OK; ++i) {
            mp_ctx* c = b->ctx[i];
            cudaStreamWaitEvent(c->stream, b->fork, 0);
            c->batch_slot = b->stage + p * n + i;
            c->n_scan = n_scan[i];
            e = cudaMemcpyAsync(c->scan_raw, b->scans + p * b->scan_floats + b->scan_off[i],
                                sizeof(float) * 3 * (size_t)n_scan[i], cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) rc = batch_err(e, "scan copy");
            if (rc == MP_OK) rc = mp_run_stages(c, MP_STAGE_ALL);
            c->batch_slot = nullptr;
            cudaEventRecord(b->join[i], c->stream);
            cudaStreamWaitEvent(b->origin, b->join[i], 0);
        }
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
    if (!b || !scans) return MP_EINVAL;
    const int p = (int)(b->steps & 1);
    B_CUDA(cudaEventSynchronize(b->done[p]));   // the launch that last read slot p
    int rc;
    for (int i = 0; i < b->n; ++i) {
        mp_ctx* c = b->ctx[i];
        if (!scans[i]) return MP_EINVAL;
        if (c->nbr_cur != (b->nbr_cur0[i] ^ p)) {
            fprintf(stderr, "mp_batch_step: instance %d was stepped outside the batch\n", i);
            return MP_EINVAL;
        }
        memcpy(b->scans + p * b->scan_floats + b->scan_off[i], scans[i], sizeof(float) * 3 * (size_t)b->n_scan[i]);
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
        mp_ctx* c = b->ctx[i];
        // later calls on the instance (mp_get_posterior, mp_step) wait for the graph
        B_CUDA(cudaStreamWaitEvent(c->stream, b->done[p], 0));
        c->n_scan = b->n_scan[i];
        c->nbr_cur ^= 1;
        c->step++;
    }
    b->steps++;
    return MP_OK;
}

int mp_batch_split(mp_batch* b, int i, int* split) {
    if (!b || !split || i < 0 || i >= b->n) return MP_EINVAL;
    *split = b->ctx[i]->lk_split > 1 ? b->ctx[i]->lk_split : 1;
    return MP_OK;
}

int mp_stream_create(void** stream) {
    if (!stream) return MP_EINVAL;
    cudaStream_t s = nullptr;
    B_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    *stream = (void*)s;
    return MP_OK;
}

int mp_stream_destroy(void* stream) {
    if (!stream) return MP_EINVAL;
    B_CUDA(cudaStreamDestroy((cudaStream_t)stream));
    return MP_OK;
}

int mp_batch_destroy(mp_batch* b) {
    if (!b) return MP_EINVAL;
    batch_free(b);
    return MP_OK;
}

}  // extern "C"
