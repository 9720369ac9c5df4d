// lsefit_batched.cuh -- every step of the fit of Section II for each series of
// a ragged batch: a small preparation launch, then one persistent launch.
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
// FP64 placement.  GB300 runs FP64 at 1/64 of the FP32 rate, and a warp
// instruction costs the same whether one lane or 32 use it.  So no FP64
// instruction runs per series inside the streaming work:
//   * the preparation launch computes every series' map constants once, one
//     series per thread;
//   * reductions stay double-float (hi, lo) pairs; a finished series is
//     queued in shared memory as pairs, and every 32 queued series (and once
//     at the end) the warp converts and solves them, one series per lane,
//     with the padded Hankel elimination;
//   * only the chunk partials of split series are combined in FP64.
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
    double eps;            // singularity threshold epsilon of the accumulation
    double* partials;      // [n_block_tasks][3*m_max+1]
    unsigned* tickets;     // [n_block_tasks], slot of a split series = its first task
    unsigned* counters;    // [0] block queue, [1] warp queue, [2] exited blocks
    double2* mapc;         // [num_series]: FP32 paths {float2(c, s), unused}; FP64 {c, s}
};

// ---------------------------------------------------------------------------
// preparation launch: clears the queue counters and split-series tickets, and
// computes the map constants of every series (one per thread).  Clearing here
// means the workspace needs no initialization and may be shared by plans of
// different layouts.
// ---------------------------------------------------------------------------
template <bool FP32MAP>
__global__ void batched_prep_kernel(BParams p) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < 3) p.counters[s] = 0u;
    if (s < p.n_block_tasks) p.tickets[s] = 0u;
    if (s >= p.num_series) return;
    double c, sc;
    const bool ok = map_constants(p.interval ? p.interval + 2 * s : nullptr, FP32MAP, c, sc);
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    double2 v;
    if (FP32MAP) {
        float2 f = ok ? make_float2((float)c, (float)sc) : make_float2(__int_as_float(0x7fc00000), 1.0f);
        v.x = __longlong_as_double(
            (long long)(((unsigned long long)__float_as_uint(f.y) << 32) | __float_as_uint(f.x)));
        v.y = 0.0;
    } else {
        v = ok ? make_double2(c, sc) : make_double2(qnan, 1.0);
    }
    p.mapc[s] = v;
    if (p.map) {
        p.map[2 * s] = ok ? c : qnan;
        p.map[2 * s + 1] = ok ? sc : qnan;
    }
}

// Map constants of series s as prepared; false if the interval was bad.
__device__ __forceinline__ bool load_map_f32(const BParams& p, int64_t s, float& c, float& sc) {
    const float2 f = *reinterpret_cast<const float2*>(p.mapc + s);
    const bool ok = !isnan(f.x);
    c = ok ? f.x : 0.0f;
    sc = ok ? f.y : 1.0f;
    return ok;
}
__device__ __forceinline__ bool load_map_f64(const BParams& p, int64_t s, double& c, double& sc) {
    const double2 v = p.mapc[s];
    const bool ok = !isnan(v.x);
    c = ok ? v.x : 0.0;
    sc = ok ? v.y : 1.0;
    return ok;
}

// ---------------------------------------------------------------------------
// queue of finished series (per warp, shared memory)
// row: word 0 = point count (int64 bits), words 1..3m+1 = accumulator totals
// (double-float pairs, or doubles for FP64 accumulation)
// ---------------------------------------------------------------------------
template <int NMAX>
struct PendLayout {
    static constexpr int kStride = 3 * NMAX + 2;
    static constexpr int kBytes = 32 * kStride * 8 + 32 * 4 * 2 + 16;
};

template <int NMAX>
struct Pend {
    unsigned long long* row;  // [32][kStride] 8-byte words
    int* sid;                 // [32] series id
    int* meta;                // [32] degree
    int* count;               // [1]
    __device__ __forceinline__ void bind(unsigned char* base) {
        row = reinterpret_cast<unsigned long long*>(base);
        sid = reinterpret_cast<int*>(base + 32 * PendLayout<NMAX>::kStride * 8);
        meta = sid + 32;
        count = meta + 32;
    }
};

__device__ __forceinline__ unsigned long long df_bits(dflt v) {
    return ((unsigned long long)__float_as_uint(v.lo) << 32) | __float_as_uint(v.hi);
}
__device__ __forceinline__ dflt bits_df(unsigned long long w) {
    dflt v;
    v.hi = __uint_as_float((unsigned)(w & 0xffffffffu));
    v.lo = __uint_as_float((unsigned)(w >> 32));
    return v;
}

// red (block reduction scratch, kBWarps x kBBlock values of 8 bytes), blk, comb, queues
constexpr size_t kRedBytes = (size_t)kBWarps * kBBlock * 8;

__host__ __device__ constexpr size_t batched_smem_bytes(int nmax) {
    return kRedBytes + 32 * 8 /* blk */ + 32 * 8 /* comb */ +
           (size_t)kBWarps * (32 * (3 * nmax + 2) * 8 + 32 * 4 * 2 + 16);
}

// The warp solves its queued series, one per lane, and empties the queue.
template <int NMAX, int ACC>
__device__ __forceinline__ void pend_solve(const BParams& p, Pend<NMAX>& q) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    const int cnt = *q.count;
    if (lane < cnt) {
        constexpr int W = PendLayout<NMAX>::kStride;
        unsigned long long* row = q.row + lane * W;
        const int m = q.meta[lane];
        const int64_t s = q.sid[lane];
        const int ns = 3 * m + 2;
        // convert this lane's row to doubles in place: S_0..S_2m, T_0..T_m
        double* sm = reinterpret_cast<double*>(row);
        sm[0] = (double)(long long)row[0];
        for (int k = 1; k < ns; ++k) {
            if (ACC != LSEFIT_ACCUM_F64) {
                const dflt v = bits_df(row[k]);
                sm[k] = (double)v.hi + (double)v.lo;
            }
        }
        double c, sc;
        bool ok;
        if (ACC == LSEFIT_ACCUM_F64) {
            ok = load_map_f64(p, s, c, sc);
        } else {
            float cf, sf;
            ok = load_map_f32(p, s, cf, sf);
            c = cf;
            sc = sf;
        }
        const int nc = p.m_max + 1;
        const int st = solve_hankel_rt<NMAX>(m, sm, sm + 2 * m + 1, c, sc, ok, p.eps,
                                             p.Xt ? p.Xt + s * nc : nullptr, p.X + s * nc, nc);
        p.status[s] = st;
        if (p.sums) {
            const double qnan = __longlong_as_double(0x7ff8000000000000ll);
            const int stride = 3 * p.m_max + 2;
            double* out = p.sums + s * stride;
            for (int k = 0; k < stride; ++k) out[k] = k < ns ? (ok ? sm[k] : qnan) : 0.0;
        }
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
    p.status[s] = LSEFIT_ERR_INVALID_ARG;
}

template <int M>
struct Unroll {
    static constexpr int value = M <= 4 ? 4 : 2;
};

// ---------------------------------------------------------------------------
// One block task: chunk `chunk` of `nch` of series s.
// ---------------------------------------------------------------------------
template <int NMAX, int DT, int ACC, int M>
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
    unsigned long long* words = reinterpret_cast<unsigned long long*>(blk);
    if constexpr (ACC == LSEFIT_ACCUM_F64) {
        double c, sc;
        const bool ok = load_map_f64(p, s, c, sc);
        AccF64<M> A;
        A.init();
        if (ok) accumulate_range_f64<M, DT, Unroll<M>::value, true>(A, p.x, p.y, b, e, tid, kBBlock, c, sc);
        block_reduce_d<kBBlock, N>([&](int a) { return A.acc[a]; }, reinterpret_cast<double*>(red), blk);
        // blk[a] (doubles) == words[a]
    } else {
        float c, sc;
        const bool ok = load_map_f32(p, s, c, sc);
        AccF32<M, ACC == LSEFIT_ACCUM_COMP> A;
        A.init();
        if (ok) accumulate_range<M, DT, ACC == LSEFIT_ACCUM_COMP, true, Unroll<M>::value>(
            A, p.x, p.y, b, e, tid, kBBlock, c, sc);
        block_reduce_df2<kBBlock, N>([&](int a) { return A.result(a); }, red, reinterpret_cast<dflt*>(blk));
    }
    // words[0..N-1] now hold this chunk's totals (visible to all threads)
    const int slot_row = PendLayout<NMAX>::kStride;
    if (nch == 1) {
        if (tid == 0) {
            const int slot = *q0.count;
            unsigned long long* row = q0.row + slot * slot_row;
            row[0] = (unsigned long long)len;
            for (int a = 0; a < N; ++a) row[a + 1] = words[a];
            q0.sid[slot] = (int)s;
            q0.meta[slot] = M;
            *q0.count = slot + 1;
        }
    } else {
        const int stride = 3 * p.m_max + 1;
        if (tid < N) {
            double v;
            if (ACC == LSEFIT_ACCUM_F64) v = blk[tid];
            else v = df_to_double(reinterpret_cast<const dflt*>(blk)[tid]);
            p.partials[(size_t)t * stride + tid] = v;
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
                unsigned long long w;
                if (ACC == LSEFIT_ACCUM_F64) {
                    w = (unsigned long long)__double_as_longlong(v);
                } else {
                    dflt d;
                    d.hi = __double2float_rn(v);
                    d.lo = __double2float_rn(v - (double)d.hi);
                    w = df_bits(d);
                }
                reinterpret_cast<unsigned long long*>(comb)[tid] = w;
            }
            __syncthreads();
            if (tid == 0) {
                const int slot = *q0.count;
                unsigned long long* row = q0.row + slot * slot_row;
                row[0] = (unsigned long long)len;
                for (int a = 0; a < N; ++a) row[a + 1] = reinterpret_cast<unsigned long long*>(comb)[a];
                q0.sid[slot] = (int)s;
                q0.meta[slot] = M;
                *q0.count = slot + 1;
                p.tickets[first] = 0u;
            }
        }
    }
    if (tid < 32) {
        __syncwarp();
        if (*q0.count == 32) pend_solve<NMAX, ACC>(p, q0);
    }
}

// ---------------------------------------------------------------------------
// One warp task: the whole of series s.
// ---------------------------------------------------------------------------
template <int NMAX, int DT, int ACC, int M>
__device__ void warp_task(const BParams& p, int64_t s, Pend<NMAX>& q) {
    constexpr int N = 3 * M + 1;
    constexpr int NP = N <= 16 ? 16 : 32;
    const int lane = threadIdx.x & 31;
    const int64_t b = p.offsets[s], e = p.offsets[s + 1];
    const int slot = *q.count;
    unsigned long long* row = q.row + slot * PendLayout<NMAX>::kStride;
    if constexpr (ACC == LSEFIT_ACCUM_F64) {
        double c, sc;
        const bool ok = load_map_f64(p, s, c, sc);
        AccF64<M> A;
        A.init();
        if (ok) accumulate_range_f64<M, DT, Unroll<M>::value, true>(A, p.x, p.y, b, e, lane, 32, c, sc);
        double v[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) v[a] = a < N ? A.acc[a] : 0.0;
        const double tot = warp_reduce_scatter_d<NP>(v);
        if (lane < N) row[lane + 1] = (unsigned long long)__double_as_longlong(tot);
    } else {
        float c, sc;
        const bool ok = load_map_f32(p, s, c, sc);
        AccF32<M, ACC == LSEFIT_ACCUM_COMP> A;
        A.init();
        if (ok) accumulate_range<M, DT, ACC == LSEFIT_ACCUM_COMP, true, Unroll<M>::value>(
            A, p.x, p.y, b, e, lane, 32, c, sc);
        dflt v[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) {
            if (a < N) {
                v[a] = A.result(a);
            } else {
                v[a].hi = 0.0f;
                v[a].lo = 0.0f;
            }
        }
        const dflt tot = warp_reduce_scatter_df<NP>(v);
        if (lane < N) row[lane + 1] = df_bits(tot);
    }
    if (lane == 0) {
        row[0] = (unsigned long long)(e - b);
        q.sid[slot] = (int)s;
        q.meta[slot] = M;
        *q.count = slot + 1;
    }
    __syncwarp();
    if (*q.count == 32) pend_solve<NMAX, ACC>(p, q);
}

template <int NMAX, int DT, int ACC>
__device__ __forceinline__ void dispatch_block(const BParams& p, int t, int4 task, int m, dflt* red,
                                               double* blk, double* comb, Pend<NMAX>& q0, int* s_last) {
    switch (m) {
        case 1: block_task<NMAX, DT, ACC, 1>(p, t, task, red, blk, comb, q0, s_last); break;
        case 2: block_task<NMAX, DT, ACC, 2>(p, t, task, red, blk, comb, q0, s_last); break;
        case 3: block_task<NMAX, DT, ACC, 3>(p, t, task, red, blk, comb, q0, s_last); break;
        case 4: block_task<NMAX, DT, ACC, 4>(p, t, task, red, blk, comb, q0, s_last); break;
        case 5: block_task<NMAX, DT, ACC, 5>(p, t, task, red, blk, comb, q0, s_last); break;
        default:
            if constexpr (NMAX > 5) {
                switch (m) {
                    case 6: block_task<NMAX, DT, ACC, 6>(p, t, task, red, blk, comb, q0, s_last); break;
                    case 7: block_task<NMAX, DT, ACC, 7>(p, t, task, red, blk, comb, q0, s_last); break;
                    default: block_task<NMAX, DT, ACC, 8>(p, t, task, red, blk, comb, q0, s_last); break;
                }
            }
            break;
    }
}

template <int NMAX, int DT, int ACC>
__device__ __forceinline__ void dispatch_warp(const BParams& p, int64_t s, int m, Pend<NMAX>& q) {
    switch (m) {
        case 1: warp_task<NMAX, DT, ACC, 1>(p, s, q); break;
        case 2: warp_task<NMAX, DT, ACC, 2>(p, s, q); break;
        case 3: warp_task<NMAX, DT, ACC, 3>(p, s, q); break;
        case 4: warp_task<NMAX, DT, ACC, 4>(p, s, q); break;
        case 5: warp_task<NMAX, DT, ACC, 5>(p, s, q); break;
        default:
            if constexpr (NMAX > 5) {
                switch (m) {
                    case 6: warp_task<NMAX, DT, ACC, 6>(p, s, q); break;
                    case 7: warp_task<NMAX, DT, ACC, 7>(p, s, q); break;
                    default: warp_task<NMAX, DT, ACC, 8>(p, s, q); break;
                }
            }
            break;
    }
}

template <int NMAX, int DT, int ACC>
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
        dispatch_block<NMAX, DT, ACC>(p, t, task, m, red, blk, comb, q0, &s_last);
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
        dispatch_warp<NMAX, DT, ACC>(p, s, m, q);
    }
    __syncwarp();
    if (*q.count > 0) pend_solve<NMAX, ACC>(p, q);
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

// Kernel for (NMAX, storage, accumulation).  The map is always applied (the
// identity map c = 0, s = 1 is exact).  Each storage/accumulation pair is
// instantiated in its own translation unit.
#define LSEFIT_BATCHED_INSTANTIATE(NAME, DT, ACC)                                  \
    batched_kernel_t NAME(int nmax) {                                              \
        return nmax <= 5 ? batched_kernel<5, DT, ACC> : batched_kernel<8, DT, ACC>; \
    }

batched_kernel_t batched_f32_naive(int nmax);
batched_kernel_t batched_f32_comp(int nmax);
batched_kernel_t batched_f32_f64(int nmax);
batched_kernel_t batched_bf16_naive(int nmax);
batched_kernel_t batched_bf16_comp(int nmax);
batched_kernel_t batched_bf16_f64(int nmax);
batched_kernel_t batched_f64_f64(int nmax);

}  // namespace lsefit
