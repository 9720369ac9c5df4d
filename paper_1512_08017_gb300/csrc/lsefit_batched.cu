// lsefit_batched.cu -- host side of the batched fit: the schedule (plan),
// workspace sizing and the launch of the persistent kernel of
// lsefit_batched.cuh.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "lsefit_batched.cuh"
#include "lsefit_host.h"

namespace lsefit {

// Threads per block of the preparation launch: one warp, because the map
// constants cost FP64 divisions, which a scheduler issues a few per hundred
// cycles, so they are spread over as many SMs as the series allow.
#ifndef LSEFIT_PREP_THREADS
#define LSEFIT_PREP_THREADS 32
#endif
constexpr int kPrepThreads = LSEFIT_PREP_THREADS;

static batched_kernel_t pick_batched(int dtype, int accum, int nmax, int basis) {
    if (basis == LSEFIT_BASIS_CHEBYSHEV) {
        if (dtype == LSEFIT_F64) return batched_f64_f64_cheb(nmax);
        if (accum == LSEFIT_ACCUM_COMP) return dtype == LSEFIT_F32 ? batched_f32_comp_cheb(nmax) : batched_bf16_comp_cheb(nmax);
        if (accum == LSEFIT_ACCUM_F64 && dtype == LSEFIT_F32) return batched_f32_f64_cheb(nmax);
        return nullptr;
    }
    if (dtype == LSEFIT_F64) return batched_f64_f64(nmax);
    if (dtype == LSEFIT_F32) {
        if (accum == LSEFIT_ACCUM_NAIVE) return batched_f32_naive(nmax);
        if (accum == LSEFIT_ACCUM_COMP) return batched_f32_comp(nmax);
        return batched_f32_f64(nmax);
    }
    if (accum == LSEFIT_ACCUM_NAIVE) return batched_bf16_naive(nmax);
    if (accum == LSEFIT_ACCUM_COMP) return batched_bf16_comp(nmax);
    return batched_bf16_f64(nmax);
}

static void resolve_tuning(const lsefit_tuning* in, lsefit_tuning* out) {
    lsefit_tuning t;
    std::memset(&t, 0, sizeof(t));
    if (in) t = *in;
    if (t.warp_max_len <= 0) t.warp_max_len = kDefaultWarpMaxLen;
    if (t.chunk_len <= 0) t.chunk_len = kDefaultChunkLen;
    if (t.chunk_len < 1024) t.chunk_len = 1024;
    t.block_threads = kBBlock;
    t.blocks_per_sm = 1;
    if (t.task_order < 1 || t.task_order > 2) t.task_order = 2;
    if (t.schedule < 1 || t.schedule > 3) t.schedule = 3;
    *out = t;
}

}  // namespace lsefit

using namespace lsefit;

extern "C" int lsefit_plan_build(const int64_t* offsets, const int32_t* degree, int64_t num_series,
                                 int m_max, const lsefit_tuning* tuning, int num_sms, lsefit_plan* plan,
                                 int32_t* block_tasks, int64_t block_cap, int32_t* warp_tasks,
                                 int64_t warp_cap) {
    if (plan == nullptr || offsets == nullptr || num_series < 0 || num_series >= (int64_t(1) << 31) ||
        m_max < 1 || m_max > LSEFIT_MAX_DEGREE || num_sms <= 0)
        return LSEFIT_ERR_INVALID_ARG;
    if (offsets[0] != 0) return LSEFIT_ERR_INVALID_ARG;
    for (int64_t s = 0; s < num_series; ++s)
        if (offsets[s + 1] < offsets[s]) return LSEFIT_ERR_INVALID_ARG;
    std::memset(plan, 0, sizeof(*plan));
    resolve_tuning(tuning, &plan->tuning);
    const int64_t wmax = plan->tuning.warp_max_len, ch = plan->tuning.chunk_len;
    std::vector<int32_t> longs, shorts;
    int64_t nbt = 0;
    int nsplit = 0;
    for (int64_t s = 0; s < num_series; ++s) {
        const int64_t len = offsets[s + 1] - offsets[s];
        if (len > wmax) {
            longs.push_back((int32_t)s);
            const int64_t nch = (len + ch - 1) / ch;
            nbt += nch;
            if (nch > 1) ++nsplit;
        } else {
            shorts.push_back((int32_t)s);
        }
    }
    if (nbt >= (int64_t(1) << 31)) return LSEFIT_ERR_INVALID_ARG;
    plan->num_series = num_series;
    plan->total_points = offsets[num_series];
    plan->n_block_tasks = (int32_t)nbt;
    plan->n_warp_tasks = (int32_t)shorts.size();
    plan->n_split_series = nsplit;
    plan->m_max = m_max;
    plan->num_sms = num_sms;
    plan->grid = 0;
    if (wmax > 0x7fffffffll) return LSEFIT_ERR_INVALID_ARG;  // a warp task's length is an int32
    if (block_cap < nbt || warp_cap < (int64_t)shorts.size() || (nbt > 0 && block_tasks == nullptr) ||
        (!shorts.empty() && warp_tasks == nullptr))
        return LSEFIT_ERR_WORKSPACE;
    auto len_of = [&](int32_t s) { return offsets[s + 1] - offsets[s]; };
    auto longer = [&](int32_t a, int32_t b) { return len_of(a) > len_of(b); };
    std::stable_sort(longs.begin(), longs.end(), longer);
    const int order = plan->tuning.task_order;
    auto cls_of = [&](int32_t s) {
        if (degree == nullptr) return 0;
        const int d = degree[s];
        return d >= 1 && d <= LSEFIT_MAX_DEGREE ? d : 0;
    };
    if (plan->tuning.schedule == 3) {
        // degree classes (invalid degrees first), longest first within a class
        auto by_class = [&](int32_t a, int32_t b) {
            const int ca = cls_of(a), cb = cls_of(b);
            return ca != cb ? ca < cb : len_of(a) > len_of(b);
        };
        std::stable_sort(shorts.begin(), shorts.end(), by_class);
    } else if (degree != nullptr && order == 2) {
        // grouped by degree (warps side by side run the same code), longest first within
        auto by_degree = [&](int32_t a, int32_t b) {
            return degree[a] != degree[b] ? degree[a] < degree[b] : len_of(a) > len_of(b);
        };
        std::stable_sort(shorts.begin(), shorts.end(), by_degree);
    } else {
        std::stable_sort(shorts.begin(), shorts.end(), longer);
    }
    {
        int32_t count[LSEFIT_MAX_DEGREE + 1] = {};
        for (int32_t s : shorts) {
            ++count[cls_of(s)];
            plan->class_points[cls_of(s)] += len_of(s);
        }
        plan->class_begin[0] = 0;
        for (int c = 0; c <= LSEFIT_MAX_DEGREE; ++c) plan->class_begin[c + 1] = plan->class_begin[c] + count[c];
    }
    int64_t t = 0;
    for (int32_t s : longs) {
        const int64_t nch = (len_of(s) + ch - 1) / ch;
        const int64_t first = t;
        for (int64_t c = 0; c < nch; ++c, ++t) {
            block_tasks[4 * t + 0] = s;
            block_tasks[4 * t + 1] = (int32_t)c;
            block_tasks[4 * t + 2] = (int32_t)nch;
            block_tasks[4 * t + 3] = (int32_t)first;
        }
    }
    plan->warp_task_len = shorts.empty() ? 0 : len_of(shorts[0]);
    for (int32_t s : shorts)
        if (len_of(s) != plan->warp_task_len) {
            plan->warp_task_len = 0;
            break;
        }
    for (size_t i = 0; i < shorts.size(); ++i) {
        const int32_t sid = shorts[i];
        const uint64_t b = (uint64_t)offsets[sid];
        warp_tasks[4 * i + 0] = sid;
        warp_tasks[4 * i + 1] = (int32_t)(uint32_t)(b & 0xffffffffu);
        warp_tasks[4 * i + 2] = (int32_t)(uint32_t)(b >> 32);
        warp_tasks[4 * i + 3] = (int32_t)len_of(sid);
    }
    return LSEFIT_OK;
}

// Workspace: queue counters | tickets [nbt] | FP64 chunk partials [nbt][3m_max+1]
// | prepared map constants [num_series] (16 bytes each).
static_assert(kCounters * sizeof(unsigned) <= kAlign, "queue counters fit the first workspace slot");
static size_t ws_tickets_off() { return kAlign; }
static size_t ws_partials_off(const lsefit_plan* plan) {
    return ws_tickets_off() + align_up((size_t)plan->n_block_tasks * sizeof(unsigned), kAlign);
}
static size_t ws_map_off(const lsefit_plan* plan) {
    return ws_partials_off(plan) +
           align_up((size_t)plan->n_block_tasks * (size_t)(3 * plan->m_max + 1) * sizeof(double), kAlign);
}
// queues of finished series: one per warp of a grid of one block per SM
static size_t ws_pend_off(const lsefit_plan* plan) {
    return ws_map_off(plan) + align_up((size_t)plan->num_series * 16, kAlign);
}
static size_t ws_pend_bytes(const lsefit_plan* plan) {
    const int nmax = plan->m_max <= 5 ? 5 : 8;
    return align_up((size_t)plan->num_sms * kBWarps * pend_warp_bytes(nmax), kAlign);
}

extern "C" size_t lsefit_batched_workspace_size(const lsefit_plan* plan) {
    if (plan == nullptr || plan->n_block_tasks < 0 || plan->num_series < 0 || plan->num_sms <= 0) return 0;
    return ws_pend_off(plan) + ws_pend_bytes(plan);
}

// Schedule 3: the persistent blocks shared out over the degree classes in
// proportion to their cost (points x relative time per point of the degree;
// block b starts on the class holding (b + 1/2) / grid of the total).  Tasks of
// an invalid degree (class 0) are only marked, so they cost nothing -- unless
// class 0 holds every point: a plan built without degrees, whose tasks are
// fitted, shares the blocks as for one class.
extern "C" int lsefit_plan_class_blocks(const lsefit_plan* plan, int grid, int32_t* cls_block) {
    if (plan == nullptr || cls_block == nullptr || grid < 1) return LSEFIT_ERR_INVALID_ARG;
    // time per point of the compensated FP32 ring at degree d relative to d = 1,
    // measured on GB300 with uniform batches (65,536 series of one degree)
    static const double kDegreeCost[kClasses] = {0.0, 1.00, 1.01, 1.05, 1.13, 1.29, 1.57, 1.86, 2.13};
    double others = 0.0;
    for (int c = 1; c < kClasses; ++c) others += (double)plan->class_points[c] * kDegreeCost[c];
    const double cost0 = others > 0.0 ? 0.0 : 1.0;
    const double total = (double)plan->class_points[0] * cost0 + others;
    int c = 0;
    double cum = (double)plan->class_points[0] * cost0;
    cls_block[0] = 0;
    for (int blk = 0; blk < grid; ++blk) {
        const double target = ((double)blk + 0.5) / (double)grid * total;
        while (c < kClasses - 1 && !(cum > target)) {
            ++c;
            cum += (double)plan->class_points[c] * kDegreeCost[c];
            cls_block[c] = blk;
        }
    }
    for (int k = c + 1; k <= kClasses; ++k) cls_block[k] = grid;
    return LSEFIT_OK;
}

extern "C" int lsefit_fit_batched(const lsefit_batch* batch, const lsefit_plan* plan, double* X,
                                  double* Xt, double* sums, double* map, int32_t* status,
                                  void* workspace, size_t workspace_bytes, lsefit_stream_t stream) {
    if (batch == nullptr || plan == nullptr || X == nullptr || status == nullptr) return LSEFIT_ERR_INVALID_ARG;
    const lsefit_batch& b = *batch;
    if (b.num_series != plan->num_series || b.m_max != plan->m_max || b.m_max < 1 ||
        b.m_max > LSEFIT_MAX_DEGREE)
        return LSEFIT_ERR_INVALID_ARG;
    if (b.dtype < LSEFIT_F64 || b.dtype > LSEFIT_BF16 || b.accum < LSEFIT_ACCUM_NAIVE ||
        b.accum > LSEFIT_ACCUM_F64)
        return LSEFIT_ERR_INVALID_ARG;
    if (b.dtype == LSEFIT_F64 && b.accum != LSEFIT_ACCUM_F64) return LSEFIT_ERR_UNSUPPORTED;
    if (b.basis != LSEFIT_BASIS_MONOMIAL && b.basis != LSEFIT_BASIS_CHEBYSHEV) return LSEFIT_ERR_INVALID_ARG;
    if (b.num_series == 0) return LSEFIT_OK;
    if (b.offsets == nullptr || b.degree == nullptr) return LSEFIT_ERR_INVALID_ARG;
    if (plan->total_points > 0 && (b.x == nullptr || b.y == nullptr)) return LSEFIT_ERR_INVALID_ARG;
    if ((plan->n_block_tasks > 0 && plan->block_tasks == nullptr) ||
        (plan->n_warp_tasks > 0 && plan->warp_tasks == nullptr))
        return LSEFIT_ERR_INVALID_ARG;
    if (workspace == nullptr || !aligned(workspace, kAlign) ||
        workspace_bytes < lsefit_batched_workspace_size(plan))
        return LSEFIT_ERR_WORKSPACE;

    BParams p;
    p.x = b.x;
    p.y = b.y;
    p.offsets = b.offsets;
    p.degree = b.degree;
    p.interval = b.interval;
    p.num_series = b.num_series;
    p.m_max = b.m_max;
    p.block_tasks = reinterpret_cast<const int4*>(plan->block_tasks);
    p.n_block_tasks = plan->n_block_tasks;
    p.warp_tasks = reinterpret_cast<const int4*>(plan->warp_tasks);
    p.n_warp_tasks = plan->n_warp_tasks;
    p.total_points = plan->total_points;
    p.sched = plan->tuning.schedule;
    for (int c = 0; c <= kClasses; ++c) p.cls_begin[c] = plan->class_begin[c];
    p.X = X;
    p.Xt = Xt;
    p.sums = sums;
    p.map = map;
    p.status = status;
    p.eps = singular_eps(b.accum);
    char* ws = static_cast<char*>(workspace);
    p.counters = reinterpret_cast<unsigned*>(ws);
    p.tickets = reinterpret_cast<unsigned*>(ws + ws_tickets_off());
    p.partials = reinterpret_cast<double*>(ws + ws_partials_off(plan));
    p.mapc = reinterpret_cast<double2*>(ws + ws_map_off(plan));
    p.pend = reinterpret_cast<unsigned char*>(ws + ws_pend_off(plan));

    const int nmax = b.m_max <= 5 ? 5 : 8;
    batched_kernel_t k = pick_batched(b.dtype, b.accum, nmax, b.basis);
    if (k == nullptr) return LSEFIT_ERR_UNSUPPORTED;
    const size_t smem = batched_smem_bytes(nmax);
    static std::mutex mu;
    static std::vector<std::pair<int, const void*>> configured;
    int dev = 0;
    const int sms = current_sm_count(&dev);
    if (sms <= 0) return LSEFIT_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lock(mu);
        const std::pair<int, const void*> key(dev, reinterpret_cast<const void*>(k));
        if (std::find(configured.begin(), configured.end(), key) == configured.end()) {
            if (cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return LSEFIT_ERR_CUDA;
            configured.push_back(key);
        }
    }
    // one block per SM: the warp rings take most of its shared memory; the
    // workspace holds the queues of exactly that many warps
    if (sms > plan->num_sms) return LSEFIT_ERR_INVALID_ARG;  // plan built for a smaller device
    int64_t grid = (int64_t)sms;
    const int64_t useful = (int64_t)plan->n_block_tasks + (plan->n_warp_tasks + kBWarps - 1) / kBWarps;
    if (useful < grid) grid = useful;
    if (grid < 1) grid = 1;
    {
        int32_t cb[kClasses + 1];
        (void)lsefit_plan_class_blocks(plan, (int)grid, cb);
        for (int c = 0; c <= kClasses; ++c) p.cls_block[c] = cb[c];
    }
    {
        const int pt = kPrepThreads;
        const int64_t items = std::max<int64_t>(std::max<int64_t>(b.num_series, plan->n_block_tasks), kCounters);
        const int64_t pb = (items + pt - 1) / pt;
        auto prep = b.accum == LSEFIT_ACCUM_F64 ? batched_prep_kernel<false> : batched_prep_kernel<true>;
        prep<<<(unsigned)pb, pt, 0, (cudaStream_t)stream>>>(p);
        if (cudaGetLastError() != cudaSuccess) return LSEFIT_ERR_CUDA;
    }
    // the persistent kernel is launched while the preparation runs (programmatic
    // dependent launch): its blocks wait for the map constants and counters
    // before their first draw
    if (launch_after_prior(k, dim3((unsigned)grid), dim3(kBBlock), smem, (cudaStream_t)stream, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return LSEFIT_ERR_CUDA;
    }
    return LSEFIT_OK;
}
