// lsefit_residuals.cu -- fitted values and residual errors of a batched fit.
//
// Section III judges a fit by its residuals e_i = y_i - f(x_i) and their sum
// of squares (Table V, the figures printed under it).  One more pass over the
// points gives, per series, SSE = sum_i r_i^2 and the orthogonality
// diagnostics (V^T r)_k = sum_i t_i^k r_i (k = 0..m), which vanish at the
// least-squares solution (the normal equations of Section II), and
// optionally the residuals themselves.  f is evaluated in the mapped basis:
// f(x_i) = sum_k Xt_k t_i^k, t_i = s (x_i - c), by Horner's rule.  For a fit
// in the Chebyshev basis (CHEB), f = sum_k Xt_k T_k(t) by Clenshaw's
// recurrence and the diagnostics are (V^T r)_k = sum_i T_k(t_i) r_i, with
// T_k(t) r following the basis recurrence from r and t r.
//
// Accumulation: FP32 per point, compensated double-float per thread
// (TwoSum per small batch), double-float warp/block reductions, FP64 chunk
// partials combined in chunk order by the block that completes a split
// series (ticket, no waiting).  FP64 data use FP64 throughout.
#include "lsefit_device.cuh"
#include "lsefit_host.h"

namespace lsefit {

constexpr int kRsBlock = 256;

struct RsParams {
    const void* x;
    const void* y;
    const int64_t* offsets;
    const int32_t* degree;
    int64_t num_series;
    int m_max;
    const double* Xt;    // [S][m_max+1]
    const double* map;   // [S][2] or null (identity)
    const int4* block_tasks;
    int n_block_tasks;
    const int4* warp_tasks;
    int n_warp_tasks;
    void* r;             // per-point residuals (FP32, or FP64 for FP64 data) or null
    double* sse;         // [S]
    double* vtr;         // [S][m_max+1] or null
    double* partials;    // [n_block_tasks][m_max+2]
    unsigned* tickets;   // [n_block_tasks]
    unsigned* counters;  // [0] block queue, [1] warp queue, [2] exited blocks
};

// Per-thread sums: a = 0 -> r^2, a = 1 + k -> t^k r (T_k(t) r for CHEB).
template <int M, bool CHEB>
struct RsAcc {
    static constexpr int N = M + 2;
    float bh[N];  // batch sums
    float hi[N], lo[N];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int a = 0; a < N; ++a) {
            bh[a] = 0.0f;
            hi[a] = 0.0f;
            lo[a] = 0.0f;
        }
    }
    __device__ __forceinline__ void add(float t, float r) {
        bh[0] = fmaf(r, r, bh[0]);
        if (CHEB) {
            const float t2 = t + t;
            float qm = r, q = t * r;  // T_0 r, T_1 r
            bh[1] += qm;
            bh[2] += q;
#pragma unroll
            for (int k = 2; k <= M; ++k) {
                const float qn = fmaf(t2, q, -qm);
                bh[1 + k] += qn;
                qm = q;
                q = qn;
            }
        } else {
            float p = r;
#pragma unroll
            for (int k = 0; k <= M; ++k) {
                bh[1 + k] += p;
                p *= t;
            }
        }
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int a = 0; a < N; ++a) {
            float s, e;
            two_sum(hi[a], bh[a], s, e);
            hi[a] = s;
            lo[a] = __fadd_rn(lo[a], e);
            bh[a] = 0.0f;
        }
    }
};

// f(t) = sum_k a_k t^k by Horner's rule, or sum_k a_k T_k(t) by Clenshaw's
// recurrence b_k = a_k + 2t b_{k+1} - b_{k+2}, f = a_0 + t b_1 - b_2.
template <int M, bool CHEB, typename F>
__device__ __forceinline__ F eval_poly(const F* a, F t) {
    if (CHEB) {
        const F t2 = t + t;
        F b1 = F(0), b2 = F(0);
#pragma unroll
        for (int k = M; k >= 1; --k) {
            const F bk = fma(t2, b1, a[k] - b2);
            b2 = b1;
            b1 = bk;
        }
        return fma(t, b1, a[0] - b2);
    }
    F v = a[M];
#pragma unroll
    for (int j = M - 1; j >= 0; --j) v = fma(v, t, a[j]);
    return v;
}

// FP32 arithmetic over [b, e): 16-byte vectors of x and y, kRsUnroll of each
// in flight per thread (the scalar head and tail of a misaligned range load
// point by point); compensated batch folded after every group of vectors.
constexpr int kRsUnroll = 4;

template <int DT, int M, bool CHEB>
__device__ __forceinline__ void rs_range_f32(const RsParams& p, int64_t s, int64_t b, int64_t e, int64_t rank,
                                             int64_t nthreads, RsAcc<M, CHEB>& A) {
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec, U = kRsUnroll;
    const int nc = p.m_max + 1;
    float coef[M + 1];
#pragma unroll
    for (int j = 0; j <= M; ++j) coef[j] = (float)p.Xt[s * nc + j];
    const float c = p.map ? (float)p.map[2 * s] : 0.0f;
    const float sc = p.map ? (float)p.map[2 * s + 1] : 1.0f;
    float* rout = static_cast<float*>(p.r);
    int64_t head, nvec;
    split_range<DT>(p.x, p.y, b, e, head, nvec);
    // residuals go out as 16-byte vectors when the output array is 16-byte aligned
    // (then every vector of points maps to PV/4 aligned float4 slots)
    const bool rvec = rout != nullptr && (reinterpret_cast<uintptr_t>(rout) & 15) == 0;
    const uint4* xv = reinterpret_cast<const uint4*>(static_cast<const char*>(p.x) + (b + head) * ES);
    const uint4* yv = reinterpret_cast<const uint4*>(static_cast<const char*>(p.y) + (b + head) * ES);
    auto feed = [&](uint4 xr, uint4 yr, int64_t i0) {
        float xs[PV], ys[PV], rr[PV];
        if (DT == LSEFIT_F32) {
            xs[0] = __uint_as_float(xr.x); xs[1] = __uint_as_float(xr.y);
            xs[2 % PV] = __uint_as_float(xr.z); xs[3 % PV] = __uint_as_float(xr.w);
            ys[0] = __uint_as_float(yr.x); ys[1] = __uint_as_float(yr.y);
            ys[2 % PV] = __uint_as_float(yr.z); ys[3 % PV] = __uint_as_float(yr.w);
        } else {
            const uint32_t xw[4] = {xr.x, xr.y, xr.z, xr.w};
            const uint32_t yw[4] = {yr.x, yr.y, yr.z, yr.w};
#pragma unroll
            for (int k = 0; k < PV / 2; ++k) {
                xs[2 * k] = bf16_lo(xw[k]); xs[2 * k + 1] = bf16_hi(xw[k]);
                ys[2 * k] = bf16_lo(yw[k]); ys[2 * k + 1] = bf16_hi(yw[k]);
            }
        }
#pragma unroll
        for (int q = 0; q < PV; ++q) {
            const float t = __fmul_rn(__fsub_rn(xs[q], c), sc);
            rr[q] = __fsub_rn(ys[q], eval_poly<M, CHEB>(coef, t));
            A.add(t, rr[q]);
        }
        if (rout) {
            if (rvec) {
#pragma unroll
                for (int q = 0; q < PV; q += 4)
                    *reinterpret_cast<float4*>(rout + i0 + q) = make_float4(rr[q], rr[q + 1], rr[q + 2], rr[q + 3]);
            } else {
#pragma unroll
                for (int q = 0; q < PV; ++q) rout[i0 + q] = rr[q];
            }
        }
    };
    const int64_t vbase = b + head;
    int64_t v = rank;
    for (; v + (U - 1) * nthreads < nvec; v += U * nthreads) {
        uint4 xr[U], yr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xr[u] = ld_stream16(xv + v + u * nthreads);
            yr[u] = ld_stream16(yv + v + u * nthreads);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) feed(xr[u], yr[u], vbase + (v + u * nthreads) * PV);
        A.fold();
    }
    for (; v < nvec; v += nthreads) {
        feed(ld_stream16(xv + v), ld_stream16(yv + v), vbase + v * PV);
        A.fold();
    }
    const int64_t tail0 = vbase + nvec * PV;
    const int64_t nscalar = head + (e - tail0);
    for (int64_t q = rank; q < nscalar; q += nthreads) {
        const int64_t i = q < head ? b + q : tail0 + (q - head);
        const float t = __fmul_rn(__fsub_rn(Elem<DT>::ld(p.x, i), c), sc);
        const float r = __fsub_rn(Elem<DT>::ld(p.y, i), eval_poly<M, CHEB>(coef, t));
        if (rout) rout[i] = r;
        A.add(t, r);
    }
    A.fold();
}

template <int M, bool CHEB>
__device__ __forceinline__ void rs_range_f64(const RsParams& p, int64_t s, int64_t b, int64_t e, int64_t rank,
                                             int64_t nthreads, double* acc) {
    const int nc = p.m_max + 1;
    double coef[M + 1];
#pragma unroll
    for (int j = 0; j <= M; ++j) coef[j] = p.Xt[s * nc + j];
    const double c = p.map ? p.map[2 * s] : 0.0;
    const double sc = p.map ? p.map[2 * s + 1] : 1.0;
    double* rout = static_cast<double*>(p.r);
    for (int64_t i = b + rank; i < e; i += nthreads) {
        const double t = sc * (Elem<LSEFIT_F64>::ld64(p.x, i) - c);
        const double r = Elem<LSEFIT_F64>::ld64(p.y, i) - eval_poly<M, CHEB>(coef, t);
        if (rout) rout[i] = r;
        acc[0] = fma(r, r, acc[0]);
        if (CHEB) {
            double qm = r, q = t * r;
            acc[1] += qm;
            acc[2] += q;
#pragma unroll
            for (int k = 2; k <= M; ++k) {
                const double qn = fma(t + t, q, -qm);
                acc[1 + k] += qn;
                qm = q;
                q = qn;
            }
        } else {
            double q = r;
#pragma unroll
            for (int k = 0; k <= M; ++k) {
                acc[1 + k] += q;
                q *= t;
            }
        }
    }
}

// Write the totals of series s (FP64), padding vtr with zeros.
__device__ __forceinline__ void rs_store(const RsParams& p, int64_t s, int M, const double* tot, bool ok) {
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    p.sse[s] = ok ? tot[0] : qnan;
    if (p.vtr) {
        const int nc = p.m_max + 1;
        for (int k = 0; k < nc; ++k) p.vtr[s * nc + k] = (ok && k <= M) ? tot[1 + k] : (k <= M ? qnan : 0.0);
    }
}

// A series whose degree is outside 1..8: SSE and the whole V^T r row are NaN.
__device__ __forceinline__ void rs_store_invalid(const RsParams& p, int64_t s) {
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    p.sse[s] = qnan;
    if (p.vtr) {
        const int nc = p.m_max + 1;
        for (int k = 0; k < nc; ++k) p.vtr[s * nc + k] = qnan;
    }
}

template <int DT, int M, bool CHEB>
__device__ void rs_block_task(const RsParams& p, int t, int4 task, dflt* red, double* red64, double* tot,
                              int* s_last) {
    constexpr int N = M + 2;
    const int tid = threadIdx.x;
    const int64_t s = task.x;
    const int chunk = task.y, nch = task.z, first = task.w;
    const int64_t b0 = p.offsets[s], e0 = p.offsets[s + 1];
    const int64_t per = ((e0 - b0 + nch - 1) / nch + 7) / 8 * 8;
    const int64_t b = min(b0 + (int64_t)chunk * per, e0), e = min(b + per, e0);
    if constexpr (DT == LSEFIT_F64) {
        double acc[N];
#pragma unroll
        for (int a = 0; a < N; ++a) acc[a] = 0.0;
        rs_range_f64<M, CHEB>(p, s, b, e, tid, kRsBlock, acc);
        block_reduce_d<kRsBlock, N>([&](int a) { return acc[a]; }, red64, tot);
    } else {
        RsAcc<M, CHEB> A;
        A.init();
        rs_range_f32<DT, M, CHEB>(p, s, b, e, tid, kRsBlock, A);
        block_reduce_df<kRsBlock, N>([&](int a) { dflt v = {A.hi[a], A.lo[a]}; return v; }, red, tot);
    }
    const bool ok = isfinite(p.Xt[s * (p.m_max + 1)]);
    if (nch == 1) {
        if (tid == 0) rs_store(p, s, M, tot, ok);
        return;
    }
    const int stride = p.m_max + 2;
    if (tid < N) {
        p.partials[(size_t)t * stride + tid] = tot[tid];
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
            tot[tid] = v;
        }
        __syncthreads();
        if (tid == 0) {
            rs_store(p, s, M, tot, ok);
            p.tickets[first] = 0u;
        }
    }
}

template <int DT, int M, bool CHEB>
__device__ void rs_warp_task(const RsParams& p, int64_t s) {
    constexpr int N = M + 2;
    const int lane = threadIdx.x & 31;
    const int64_t b = p.offsets[s], e = p.offsets[s + 1];
    double tot[N];
    if constexpr (DT == LSEFIT_F64) {
        double acc[N];
#pragma unroll
        for (int a = 0; a < N; ++a) acc[a] = 0.0;
        rs_range_f64<M, CHEB>(p, s, b, e, lane, 32, acc);
#pragma unroll
        for (int a = 0; a < N; ++a) tot[a] = warp_reduce_d(acc[a]);
    } else {
        RsAcc<M, CHEB> A;
        A.init();
        rs_range_f32<DT, M, CHEB>(p, s, b, e, lane, 32, A);
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const dflt v = {A.hi[a], A.lo[a]};
            tot[a] = df_to_double(warp_reduce_df(v));
        }
    }
    if (lane == 0) rs_store(p, s, M, tot, isfinite(p.Xt[s * (p.m_max + 1)]));
}

template <int DT, bool CHEB>
__global__ void __launch_bounds__(kRsBlock) residuals_kernel(__grid_constant__ const RsParams p) {
    __shared__ int s_task;
    __shared__ int s_last;
    __shared__ dflt red[(kRsBlock / 32) * kRsBlock];
    __shared__ double tot[16];
    const int tid = threadIdx.x, lane = tid & 31;
    double* red64 = reinterpret_cast<double*>(red);
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(&p.counters[0], 1u);
        __syncthreads();
        const int t = s_task;
        __syncthreads();
        if (t >= p.n_block_tasks) break;
        const int4 task = p.block_tasks[t];
        const int m = p.degree[task.x];
        // a degree above m_max has no coefficient row of its length: invalid
        switch (m <= p.m_max ? m : 0) {
            case 1: rs_block_task<DT, 1, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            case 2: rs_block_task<DT, 2, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            case 3: rs_block_task<DT, 3, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            case 4: rs_block_task<DT, 4, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            case 5: rs_block_task<DT, 5, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            case 6: rs_block_task<DT, 6, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            case 7: rs_block_task<DT, 7, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            case 8: rs_block_task<DT, 8, CHEB>(p, t, task, red, red64, tot, &s_last); break;
            default:
                if (tid == 0 && task.y == 0) rs_store_invalid(p, task.x);
                break;
        }
        __syncthreads();
    }
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&p.counters[1], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= p.n_warp_tasks) break;
        const int64_t s = p.warp_tasks[t].x;
        const int m = p.degree[s];
        switch (m <= p.m_max ? m : 0) {
            case 1: rs_warp_task<DT, 1, CHEB>(p, s); break;
            case 2: rs_warp_task<DT, 2, CHEB>(p, s); break;
            case 3: rs_warp_task<DT, 3, CHEB>(p, s); break;
            case 4: rs_warp_task<DT, 4, CHEB>(p, s); break;
            case 5: rs_warp_task<DT, 5, CHEB>(p, s); break;
            case 6: rs_warp_task<DT, 6, CHEB>(p, s); break;
            case 7: rs_warp_task<DT, 7, CHEB>(p, s); break;
            case 8: rs_warp_task<DT, 8, CHEB>(p, s); break;
            default:
                if (lane == 0) rs_store_invalid(p, s);
                break;
        }
    }
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

__global__ void residuals_prep_kernel(unsigned* counters, unsigned* tickets, int n_block_tasks) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3) counters[i] = 0u;
    if (i < n_block_tasks) tickets[i] = 0u;
}

}  // namespace lsefit

using namespace lsefit;

// Workspace: counters | tickets [nbt] | FP64 partials [nbt][m_max+2].
extern "C" size_t lsefit_residuals_workspace_size(const lsefit_plan* plan) {
    if (plan == nullptr || plan->n_block_tasks < 0 || plan->m_max < 1) return 0;
    const size_t nbt = (size_t)plan->n_block_tasks;
    return kAlign + align_up(nbt * sizeof(unsigned), kAlign) + align_up(nbt * (plan->m_max + 2) * sizeof(double), kAlign);
}

extern "C" int lsefit_residuals(const lsefit_batch* batch, const lsefit_plan* plan, const double* Xt,
                                const double* map, void* r, double* sse, double* vtr, void* workspace,
                                size_t workspace_bytes, lsefit_stream_t stream) {
    if (batch == nullptr || plan == nullptr || Xt == nullptr || sse == nullptr) return LSEFIT_ERR_INVALID_ARG;
    const lsefit_batch& b = *batch;
    if (b.num_series != plan->num_series || b.m_max != plan->m_max || b.m_max < 1 || b.m_max > LSEFIT_MAX_DEGREE)
        return LSEFIT_ERR_INVALID_ARG;
    if (b.dtype < LSEFIT_F64 || b.dtype > LSEFIT_BF16) return LSEFIT_ERR_INVALID_ARG;
    if (b.basis != LSEFIT_BASIS_MONOMIAL && b.basis != LSEFIT_BASIS_CHEBYSHEV) return LSEFIT_ERR_INVALID_ARG;
    if (b.num_series == 0) return LSEFIT_OK;
    if (b.offsets == nullptr || b.degree == nullptr) return LSEFIT_ERR_INVALID_ARG;
    if (plan->total_points > 0 && (b.x == nullptr || b.y == nullptr)) return LSEFIT_ERR_INVALID_ARG;
    if (workspace == nullptr || !aligned(workspace, kAlign) ||
        workspace_bytes < lsefit_residuals_workspace_size(plan))
        return LSEFIT_ERR_WORKSPACE;
    RsParams p;
    p.x = b.x;
    p.y = b.y;
    p.offsets = b.offsets;
    p.degree = b.degree;
    p.num_series = b.num_series;
    p.m_max = b.m_max;
    p.Xt = Xt;
    p.map = map;
    p.block_tasks = reinterpret_cast<const int4*>(plan->block_tasks);
    p.n_block_tasks = plan->n_block_tasks;
    p.warp_tasks = reinterpret_cast<const int4*>(plan->warp_tasks);
    p.n_warp_tasks = plan->n_warp_tasks;
    p.r = r;
    p.sse = sse;
    p.vtr = vtr;
    char* ws = static_cast<char*>(workspace);
    p.counters = reinterpret_cast<unsigned*>(ws);
    p.tickets = reinterpret_cast<unsigned*>(ws + kAlign);
    p.partials = reinterpret_cast<double*>(ws + kAlign + align_up((size_t)plan->n_block_tasks * sizeof(unsigned), kAlign));
    const int items = plan->n_block_tasks > 3 ? plan->n_block_tasks : 3;
    residuals_prep_kernel<<<(items + 255) / 256, 256, 0, (cudaStream_t)stream>>>(p.counters, p.tickets,
                                                                               plan->n_block_tasks);
    if (cudaGetLastError() != cudaSuccess) return LSEFIT_ERR_CUDA;
    const bool cheb = b.basis == LSEFIT_BASIS_CHEBYSHEV;
    auto k = b.dtype == LSEFIT_F64 ? (cheb ? residuals_kernel<LSEFIT_F64, true> : residuals_kernel<LSEFIT_F64, false>)
             : b.dtype == LSEFIT_F32 ? (cheb ? residuals_kernel<LSEFIT_F32, true> : residuals_kernel<LSEFIT_F32, false>)
                                     : (cheb ? residuals_kernel<LSEFIT_BF16, true> : residuals_kernel<LSEFIT_BF16, false>);
    int dev = 0;
    const int sms = current_sm_count(&dev);
    if (sms <= 0) return LSEFIT_ERR_CUDA;
    const int occ = occupancy_blocks(reinterpret_cast<const void*>(k), kRsBlock, 0);
    int64_t grid = (int64_t)sms * occ;
    const int64_t useful = (int64_t)plan->n_block_tasks + (plan->n_warp_tasks + 7) / 8;
    if (useful < grid) grid = useful;
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, kRsBlock, 0, (cudaStream_t)stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? LSEFIT_OK : LSEFIT_ERR_CUDA;
}
