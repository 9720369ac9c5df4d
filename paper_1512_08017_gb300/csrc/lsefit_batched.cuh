// lsefit_batched.cuh -- every step of the fit of Section II for each series of
// a ragged batch, in one persistent launch.
//
// Schedule (built on the host by lsefit_plan_build, replayed as is):
//   * block tasks: series longer than warp_max_len, cut into chunks of about
//     chunk_len points; one block reduces one chunk.  A series of one chunk
//     is finished by its block; otherwise each chunk's block stores an FP64
//     partial and takes a ticket, and the block that completes the series
//     adds the partials in chunk order (no block ever waits for another);
//   * warp tasks: the shorter series, longest first; one warp reduces one
//     series.
// Persistent blocks take block tasks from an atomic queue until it is
// empty, then each warp takes warp tasks from a second queue.
//
// Solving: the finished series of a warp (its own, or, for warp 0, those
// completed by its block) are queued in shared memory with their FP64 sums;
// every 32 of them, and once at the end, the warp solves them one per lane
// with the padded Hankel elimination (FP64 throughput is spent on 32 systems
// per instruction instead of one).
#pragma once

#include "lsefit_device.cuh"

namespace lsefit {

constexpr int kBBlock = 256;
constexpr int kBWarps = kBBlock / 32;
constexpr int kDefaultWarpMaxLen = 8192;
constexpr int kDefaultChunkLen = 65536;

struct BParams {
    const void* x;
    const void* y;
    const int64_t* offsets;
    const int32_t* degree;
    const double* interval;
    int64_t num_series;
    int m_max;
    const int4* block_tasks;
    int n_block_tasks;
    const int32_t* warp_tasks;
    int n_warp_tasks;
    double* X;
    double* Xt;
    double* sums;
    double* map;
    int32_t* status;
    double* partials;      // [n_block_tasks][3*m_max+1]
    unsigned* tickets;     // [n_block_tasks], slot of a split series = its first task
    unsigned* counters;    // [0] block queue, [1] warp queue, [2] exited blocks
};

// Shared-memory layout of one warp's queue of finished series.
template <int NMAX>
struct PendLayout {
    static constexpr int kSums = 3 * NMAX + 2;
    static constexpr int kStride = kSums + 3;  // sums, c, s, (pad)
    static constexpr int kBytes = 32 * kStride * 8 + 32 * 4 * 2 + 16;
};

template <int NMAX>
struct Pend {
    double* row;  // [32][kStride]: S_0..S_2m T_0..T_m | c | s
    int* sid;     // [32] series id
    int* meta;    // [32] m | (map ok << 8)
    int* count;   // [1]
    __device__ __forceinline__ void bind(unsigned char* base) {
        row = reinterpret_cast<double*>(base);
        sid = reinterpret_cast<int*>(base + 32 * PendLayout<NMAX>::kStride * 8);
        meta = sid + 32;
        count = meta + 32;
    }
};

// red (block reduction scratch, kBWarps x kBBlock values of 8 bytes), blk, comb, queues
constexpr size_t kRedBytes = (size_t)kBWarps * kBBlock * 8;

__host__ __device__ constexpr size_t batched_smem_bytes(int nmax) {
    return kRedBytes + 32 * 8 /* blk */ + 32 * 8 /* comb */ +
           (size_t)kBWarps * (32 * (3 * nmax + 5) * 8 + 32 * 4 * 2 + 16);
}

// Map constants of series s (FP32-rounded unless the arithmetic is FP64).
__device__ __forceinline__ bool series_map(const BParams& p, int64_t s, bool fp32, double& c, double& sc) {
    return map_constants(p.interval ? p.interval + 2 * s : nullptr, fp32, c, sc);
}

// Queue a finished series (called by one thread).  sums0..: S_0..S_2m T_0..T_m.
template <int NMAX>
__device__ __forceinline__ void pend_push(const BParams& p, Pend<NMAX>& q, int64_t s, int m,
                                          const double* sm, bool ok, double c, double sc) {
    const int slot = *q.count;
    double* row = q.row + slot * PendLayout<NMAX>::kStride;
    const int ns = 3 * m + 2;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int k = 0; k < ns; ++k) row[k] = sm[k];
    row[PendLayout<NMAX>::kSums] = c;
    row[PendLayout<NMAX>::kSums + 1] = sc;
    q.sid[slot] = (int)s;
    q.meta[slot] = m | (ok ? 256 : 0);
    *q.count = slot + 1;
    if (p.sums) {
        const int stride = 3 * p.m_max + 2;
        double* out = p.sums + s * stride;
        for (int k = 0; k < stride; ++k) out[k] = k < ns ? (ok ? sm[k] : qnan) : 0.0;
    }
    if (p.map) {
        p.map[2 * s] = ok ? c : qnan;
        p.map[2 * s + 1] = ok ? sc : qnan;
    }
}

// The warp solves its queued series, one per lane, and empties the queue.
template <int NMAX>
__device__ __forceinline__ void pend_solve(const BParams& p, Pend<NMAX>& q) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    const int cnt = *q.count;
    if (lane < cnt) {
        const double* row = q.row + lane * PendLayout<NMAX>::kStride;
        const int meta = q.meta[lane];
        const int m = meta & 255;
        const bool ok = (meta >> 8) & 1;
        const int64_t s = q.sid[lane];
        const int nc = p.m_max + 1;
        const int st = solve_hankel_rt<NMAX>(m, row, row + 2 * m + 1, row[PendLayout<NMAX>::kSums],
                                             row[PendLayout<NMAX>::kSums + 1], ok,
                                             p.Xt ? p.Xt + s * nc : nullptr, p.X + s * nc, nc);
        p.status[s] = st;
    }
    __syncwarp();
    if (lane == 0) *q.count = 0;
    __syncwarp();
}

// Status and NaN row of a series that is not fitted at all (bad degree).
__device__ __forceinline__ void mark_invalid(const BParams& p, int64_t s) {
    const int nc = p.m_max + 1;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int i = 0; i < nc; ++i) {
        p.X[s * nc + i] = qnan;
        if (p.Xt) p.Xt[s * nc + i] = qnan;
    }
    if (p.sums) {
        for (int k = 0; k < 3 * p.m_max + 2; ++k) p.sums[s * (3 * p.m_max + 2) + k] = qnan;
    }
    if (p.map) {
        p.map[2 * s] = qnan;
        p.map[2 * s + 1] = qnan;
    }
    p.status[s] = LSEFIT_ERR_INVALID_ARG;
}

template <int M>
struct Unroll {
    static constexpr int value = M <= 4 ? 4 : 2;
};

// ---------------------------------------------------------------------------
// One block task: chunk `chunk` of `nch` of series s.
// ---------------------------------------------------------------------------
template <int NMAX, int DT, int ACC, bool MAP, int M>
__device__ void block_task(const BParams& p, int t, int4 task, dflt* red, double* blk, double* comb,
                           Pend<NMAX>& q0, int* s_last) {
    constexpr int N = 3 * M + 1;
    const int tid = threadIdx.x;
    const int64_t s = task.x;
    const int chunk = task.y, nch = task.z, first = task.w;
    const int64_t b0 = p.offsets[s], e0 = p.offsets[s + 1];
    const int64_t len = e0 - b0;
    const int64_t per = ((len + nch - 1) / nch + 7) / 8 * 8;
    const int64_t b = min(b0 + (int64_t)chunk * per, e0);
    const int64_t e = min(b + per, e0);
    double c, sc;
    const bool ok = series_map(p, s, ACC != LSEFIT_ACCUM_F64, c, sc);
    if constexpr (ACC == LSEFIT_ACCUM_F64) {
        AccF64<M> A;
        A.init();
        accumulate_range_f64<M, DT, Unroll<M>::value, MAP>(A, p.x, p.y, b, e, tid, kBBlock, c, sc);
        block_reduce_d<kBBlock, N>([&](int a) { return A.acc[a]; }, reinterpret_cast<double*>(red), blk);
    } else {
        AccF32<M, ACC == LSEFIT_ACCUM_COMP> A;
        A.init();
        accumulate_range<M, DT, ACC == LSEFIT_ACCUM_COMP, MAP, Unroll<M>::value>(
            A, p.x, p.y, b, e, tid, kBBlock, (float)c, (float)sc);
        block_reduce_df<kBBlock, N>([&](int a) { return A.result(a); }, red, blk);
    }
    // blk[0..N-1] now holds this chunk's sums (visible to all threads)
    if (nch == 1) {
        if (tid == 0) {
            comb[0] = (double)len;
            for (int a = 0; a < N; ++a) comb[a + 1] = blk[a];
            pend_push<NMAX>(p, q0, s, M, comb, ok, c, sc);
        }
    } else {
        const int stride = 3 * p.m_max + 1;
        if (tid < N) {
            p.partials[(size_t)t * stride + tid] = blk[tid];
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) *s_last = (atomicAdd(&p.tickets[first], 1u) == (unsigned)(nch - 1));
        __syncthreads();
        if (*s_last) {
            __threadfence();
            if (tid < N) {
                double v = 0.0;
                for (int k = 0; k < nch; ++k) v += __ldcg(p.partials + (size_t)(first + k) * stride + tid);
                comb[tid + 1] = v;
            }
            __syncthreads();
            if (tid == 0) {
                comb[0] = (double)len;
                pend_push<NMAX>(p, q0, s, M, comb, ok, c, sc);
                p.tickets[first] = 0u;
            }
        }
    }
    if (tid < 32) {
        __syncwarp();
        if (*q0.count == 32) pend_solve<NMAX>(p, q0);
    }
}

// ---------------------------------------------------------------------------
// One warp task: the whole of series s.
// ---------------------------------------------------------------------------
template <int NMAX, int DT, int ACC, bool MAP, int M>
__device__ void warp_task(const BParams& p, int64_t s, Pend<NMAX>& q) {
    constexpr int N = 3 * M + 1;
    const int lane = threadIdx.x & 31;
    const int64_t b = p.offsets[s], e = p.offsets[s + 1];
    double c, sc;
    const bool ok = series_map(p, s, ACC != LSEFIT_ACCUM_F64, c, sc);
    double tot[N + 1];
    tot[0] = (double)(e - b);
    if constexpr (ACC == LSEFIT_ACCUM_F64) {
        AccF64<M> A;
        A.init();
        accumulate_range_f64<M, DT, Unroll<M>::value, MAP>(A, p.x, p.y, b, e, lane, 32, c, sc);
#pragma unroll
        for (int a = 0; a < N; ++a) tot[a + 1] = warp_reduce_d(A.acc[a]);
    } else {
        AccF32<M, ACC == LSEFIT_ACCUM_COMP> A;
        A.init();
        accumulate_range<M, DT, ACC == LSEFIT_ACCUM_COMP, MAP, Unroll<M>::value>(
            A, p.x, p.y, b, e, lane, 32, (float)c, (float)sc);
#pragma unroll
        for (int a = 0; a < N; ++a) tot[a + 1] = df_to_double(warp_reduce_df(A.result(a)));
    }
    if (lane == 0) pend_push<NMAX>(p, q, s, M, tot, ok, c, sc);
    __syncwarp();
    if (*q.count == 32) pend_solve<NMAX>(p, q);
}

template <int NMAX, int DT, int ACC, bool MAP>
__device__ __forceinline__ void dispatch_block(const BParams& p, int t, int4 task, int m, dflt* red,
                                               double* blk, double* comb, Pend<NMAX>& q0, int* s_last) {
    switch (m) {
        case 1: block_task<NMAX, DT, ACC, MAP, 1>(p, t, task, red, blk, comb, q0, s_last); break;
        case 2: block_task<NMAX, DT, ACC, MAP, 2>(p, t, task, red, blk, comb, q0, s_last); break;
        case 3: block_task<NMAX, DT, ACC, MAP, 3>(p, t, task, red, blk, comb, q0, s_last); break;
        case 4: block_task<NMAX, DT, ACC, MAP, 4>(p, t, task, red, blk, comb, q0, s_last); break;
        case 5: block_task<NMAX, DT, ACC, MAP, 5>(p, t, task, red, blk, comb, q0, s_last); break;
        default:
            if constexpr (NMAX > 5) {
                switch (m) {
                    case 6: block_task<NMAX, DT, ACC, MAP, 6>(p, t, task, red, blk, comb, q0, s_last); break;
                    case 7: block_task<NMAX, DT, ACC, MAP, 7>(p, t, task, red, blk, comb, q0, s_last); break;
                    default: block_task<NMAX, DT, ACC, MAP, 8>(p, t, task, red, blk, comb, q0, s_last); break;
                }
            }
            break;
    }
}

template <int NMAX, int DT, int ACC, bool MAP>
__device__ __forceinline__ void dispatch_warp(const BParams& p, int64_t s, int m, Pend<NMAX>& q) {
    switch (m) {
        case 1: warp_task<NMAX, DT, ACC, MAP, 1>(p, s, q); break;
        case 2: warp_task<NMAX, DT, ACC, MAP, 2>(p, s, q); break;
        case 3: warp_task<NMAX, DT, ACC, MAP, 3>(p, s, q); break;
        case 4: warp_task<NMAX, DT, ACC, MAP, 4>(p, s, q); break;
        case 5: warp_task<NMAX, DT, ACC, MAP, 5>(p, s, q); break;
        default:
            if constexpr (NMAX > 5) {
                switch (m) {
                    case 6: warp_task<NMAX, DT, ACC, MAP, 6>(p, s, q); break;
                    case 7: warp_task<NMAX, DT, ACC, MAP, 7>(p, s, q); break;
                    default: warp_task<NMAX, DT, ACC, MAP, 8>(p, s, q); break;
                }
            }
            break;
    }
}

template <int NMAX, int DT, int ACC, bool MAP>
__global__ void __launch_bounds__(kBBlock, NMAX <= 5 ? 2 : 1) batched_kernel(BParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_task;
    __shared__ int s_last;
    dflt* red = reinterpret_cast<dflt*>(smem);
    double* blk = reinterpret_cast<double*>(smem + kRedBytes);
    double* comb = blk + 32;
    unsigned char* pend_base = reinterpret_cast<unsigned char*>(comb + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    Pend<NMAX> q;
    q.bind(pend_base + warp * PendLayout<NMAX>::kBytes);
    Pend<NMAX> q0;
    q0.bind(pend_base);
    if (lane == 0) *q.count = 0;
    __syncthreads();

    // phase 1: block tasks
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(&p.counters[0], 1u);
        __syncthreads();
        const int t = s_task;
        __syncthreads();
        if (t >= p.n_block_tasks) break;
        const int4 task = p.block_tasks[t];
        const int m = p.degree[task.x];
        if (m < 1 || m > p.m_max || m > NMAX) {
            if (tid == 0 && task.y == 0) mark_invalid(p, task.x);
            continue;
        }
        dispatch_block<NMAX, DT, ACC, MAP>(p, t, task, m, red, blk, comb, q0, &s_last);
    }
    // phase 2: warp tasks
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&p.counters[1], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= p.n_warp_tasks) break;
        const int64_t s = p.warp_tasks[t];
        const int m = p.degree[s];
        if (m < 1 || m > p.m_max || m > NMAX) {
            if (lane == 0) mark_invalid(p, s);
            continue;
        }
        dispatch_warp<NMAX, DT, ACC, MAP>(p, s, m, q);
    }
    if (*q.count > 0) pend_solve<NMAX>(p, q);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&p.counters[2], 1u) == gridDim.x - 1) {
            p.counters[0] = 0u;
            p.counters[1] = 0u;
            p.counters[2] = 0u;
        }
    }
}

typedef void (*batched_kernel_t)(BParams);

// Kernel for (NMAX, storage, accumulation); the map is always applied (the
// identity map c = 0, s = 1 is exact).  Each storage/accumulation pair is
// instantiated in its own translation unit.
#define LSEFIT_BATCHED_INSTANTIATE(NAME, DT, ACC)                                  \
    batched_kernel_t NAME(int nmax) {                                              \
        return nmax <= 5 ? batched_kernel<5, DT, ACC, true> : batched_kernel<8, DT, ACC, true>; \
    }

batched_kernel_t batched_f32_naive(int nmax);
batched_kernel_t batched_f32_comp(int nmax);
batched_kernel_t batched_f32_f64(int nmax);
batched_kernel_t batched_bf16_naive(int nmax);
batched_kernel_t batched_bf16_comp(int nmax);
batched_kernel_t batched_bf16_f64(int nmax);
batched_kernel_t batched_f64_f64(int nmax);

}  // namespace lsefit
