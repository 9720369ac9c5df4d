// lsefit_autotune.cu -- the autotuner of the batched schedule: every
// candidate tuning is turned into a plan of the caller's layout, run on the
// caller's batch with CUDA events around it, and the fastest is returned.
//
// The best split of a batch into block tasks and warp tasks, the chunk
// length and the way warps draw their tasks depend on the length and degree
// distribution of the batch and on the device, so they are measured rather
// than modelled.  The library allocates no device memory here either: the
// caller passes device buffers for the candidates' task arrays, the batched
// workspace and the fit's outputs (sized by lsefit_plan_autotune_sizes).
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "lsefit.h"
#include "lsefit_host.h"

namespace {

// Built-in candidates: the three ways warps draw warp tasks with every series
// a warp task, and the degree-class schedule with block tasks for series
// above 4,096 or 65,536 points cut into chunks of 65,536 or 262,144.
const lsefit_tuning* builtin_candidates(int* count) {
    static lsefit_tuning c[LSEFIT_AUTOTUNE_MAX_CANDIDATES];
    static int n = 0;
    static bool init = false;
    if (!init) {
        std::memset(c, 0, sizeof(c));
        for (int sched = 1; sched <= 3; ++sched) {
            c[n].warp_max_len = 1 << 20;
            c[n].schedule = sched;
            ++n;
        }
        const int wmax[2] = {4096, 65536};
        const int chunk[2] = {65536, 262144};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                c[n].warp_max_len = wmax[a];
                c[n].chunk_len = chunk[b];
                c[n].schedule = 3;
                ++n;
            }
        init = true;
    }
    *count = n;
    return c;
}

struct HostPlan {
    lsefit_plan plan;
    std::vector<int32_t> tasks;  // block tasks, then warp tasks (4 int32 each)
};

int build_host_plan(const int64_t* offsets, const int32_t* degree, int64_t num_series, int m_max,
                    const lsefit_tuning* tuning, int num_sms, HostPlan* out) {
    int rc = lsefit_plan_build(offsets, degree, num_series, m_max, tuning, num_sms, &out->plan, nullptr, 0,
                               nullptr, 0);
    if (rc != LSEFIT_OK && rc != LSEFIT_ERR_WORKSPACE) return rc;
    const int64_t nb = out->plan.n_block_tasks, nw = out->plan.n_warp_tasks;
    out->tasks.assign((size_t)(4 * (nb + nw)) + 4, 0);
    return lsefit_plan_build(offsets, degree, num_series, m_max, tuning, num_sms, &out->plan, out->tasks.data(),
                             nb, out->tasks.data() + 4 * nb, nw);
}

}  // namespace

using namespace lsefit;

extern "C" int lsefit_autotune_candidates(lsefit_tuning* out, int cap) {
    int n = 0;
    const lsefit_tuning* c = builtin_candidates(&n);
    if (out != nullptr)
        for (int i = 0; i < n && i < cap; ++i) out[i] = c[i];
    return n;
}

extern "C" int lsefit_plan_autotune_sizes(const int64_t* offsets_host, const int32_t* degree_host,
                                          int64_t num_series, int m_max, const lsefit_tuning* candidates,
                                          int n_candidates, int num_sms, int64_t* task_ints,
                                          size_t* workspace_bytes) {
    if (offsets_host == nullptr || task_ints == nullptr || workspace_bytes == nullptr || num_sms <= 0)
        return LSEFIT_ERR_INVALID_ARG;
    if (candidates == nullptr) candidates = builtin_candidates(&n_candidates);
    if (n_candidates < 1 || n_candidates > LSEFIT_AUTOTUNE_MAX_CANDIDATES) return LSEFIT_ERR_INVALID_ARG;
    int64_t ints = 4;
    size_t ws = 0;
    for (int i = 0; i < n_candidates; ++i) {
        lsefit_plan plan;
        const int rc = lsefit_plan_build(offsets_host, degree_host, num_series, m_max, &candidates[i], num_sms,
                                         &plan, nullptr, 0, nullptr, 0);
        if (rc != LSEFIT_OK && rc != LSEFIT_ERR_WORKSPACE) return rc;
        const int64_t need = 4 * ((int64_t)plan.n_block_tasks + plan.n_warp_tasks);
        if (need > ints) ints = need;
        const size_t w = lsefit_batched_workspace_size(&plan);
        if (w > ws) ws = w;
    }
    *task_ints = ints;
    *workspace_bytes = ws;
    return LSEFIT_OK;
}

extern "C" int lsefit_plan_autotune(const lsefit_batch* batch, const int64_t* offsets_host,
                                    const int32_t* degree_host, const lsefit_tuning* candidates,
                                    int n_candidates, int reps, int32_t* tasks_device, int64_t task_ints,
                                    void* workspace, size_t workspace_bytes, double* X, int32_t* status,
                                    lsefit_stream_t stream, lsefit_tuning* best, float* ms_per_candidate) {
    if (batch == nullptr || offsets_host == nullptr || tasks_device == nullptr || workspace == nullptr ||
        X == nullptr || status == nullptr || best == nullptr || reps < 1)
        return LSEFIT_ERR_INVALID_ARG;
    if (candidates == nullptr) candidates = builtin_candidates(&n_candidates);
    if (n_candidates < 1 || n_candidates > LSEFIT_AUTOTUNE_MAX_CANDIDATES) return LSEFIT_ERR_INVALID_ARG;
    if (((uintptr_t)tasks_device & 15) != 0) return LSEFIT_ERR_WORKSPACE;
    int dev = 0;
    const int sms = current_sm_count(&dev);
    if (sms <= 0) return LSEFIT_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t cs = nullptr;  // private stream the candidates' fits are captured on
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        (void)cudaGetLastError();
        return LSEFIT_ERR_CUDA;
    }
    int rc = LSEFIT_OK;
    float best_ms = -1.0f;
    for (int i = 0; i < n_candidates && rc == LSEFIT_OK; ++i) {
        HostPlan hp;
        rc = build_host_plan(offsets_host, degree_host, batch->num_series, batch->m_max, &candidates[i], sms, &hp);
        if (rc != LSEFIT_OK) break;
        const int64_t nb = hp.plan.n_block_tasks, nw = hp.plan.n_warp_tasks;
        if (4 * (nb + nw) > task_ints || lsefit_batched_workspace_size(&hp.plan) > workspace_bytes) {
            rc = LSEFIT_ERR_WORKSPACE;
            break;
        }
        // the host task arrays must outlive the copy: wait for it before they go
        if (nb + nw > 0 &&
            (cudaMemcpyAsync(tasks_device, hp.tasks.data(), (size_t)(4 * (nb + nw)) * sizeof(int32_t),
                             cudaMemcpyHostToDevice, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess)) {
            rc = LSEFIT_ERR_CUDA;
            break;
        }
        hp.plan.block_tasks = tasks_device;
        hp.plan.warp_tasks = tasks_device + 4 * nb;
        rc = lsefit_fit_batched(batch, &hp.plan, X, nullptr, nullptr, nullptr, status, workspace, workspace_bytes,
                                stream);  // warm-up (also sets the kernel's attributes outside the capture)
        if (rc != LSEFIT_OK) break;
        // Time replays of the fit captured in a CUDA graph, the way a caller that
        // replays graphs runs it: timed as plain back-to-back calls, the schedules
        // can differ by less than the noise while their graph replays do not.
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = LSEFIT_ERR_CUDA;
            break;
        }
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = LSEFIT_ERR_CUDA;
            break;
        }
        rc = lsefit_fit_batched(batch, &hp.plan, X, nullptr, nullptr, nullptr, status, workspace, workspace_bytes,
                                (lsefit_stream_t)cs);
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (rc == LSEFIT_OK && (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess))
            rc = LSEFIT_ERR_CUDA;
        float ms = 0.0f;
        if (rc == LSEFIT_OK) {
            if (cudaGraphLaunch(exec, st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess) rc = LSEFIT_ERR_CUDA;
            for (int r = 0; r < reps && rc == LSEFIT_OK; ++r)
                if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = LSEFIT_ERR_CUDA;
            if (rc == LSEFIT_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = LSEFIT_ERR_CUDA;
        }
        if (exec != nullptr) cudaGraphExecDestroy(exec);
        if (graph != nullptr) cudaGraphDestroy(graph);
        if (rc != LSEFIT_OK) break;
        ms /= (float)reps;
        if (ms_per_candidate != nullptr) ms_per_candidate[i] = ms;
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            *best = hp.plan.tuning;
        }
    }
    if (rc == LSEFIT_ERR_CUDA) (void)cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    return rc;
}

extern "C" int lsefit_driver_version(void) {
    int v = 0;
    if (cudaDriverGetVersion(&v) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return v;
}
