// lsefit_backward.cu -- adjoint of the batched fit.
//
// The fit solves A Xt = B (Section II: A[j][k] = S_{j+k}, B[j] = T_j) on the
// mapped abscissae t = s (x - c) and returns X = M Xt.  For a loss L(X) with
// gX = dL/dX, the chain rule through the normal equations gives
//   gt = M^T gX,  A lambda = gt  (A symmetric),
//   dL/dT_j = lambda_j,  dL/dS_p = -sum_{j+k=p} lambda_j Xt_k,
// and, through T_j = sum_i t_i^j y_i and S_p = sum_i t_i^p,
//   dL/dy_i = lambda(t_i),
//   dL/dt_i = lambda'(t_i) (y_i - f(t_i)) - lambda(t_i) f'(t_i),  f = sum_k Xt_k t^k,
//   dL/dx_i = s dL/dt_i           (c and s held fixed).
// Launch 1 solves for lambda, one series per thread (FP64, padded
// elimination).  Launch 2 streams the points once more with the forward
// plan's tasks, recomputing t and the polynomial values by Horner's rule
// with derivative (packed FP32 pairs; FP64 for FP64 data).  Launch 2 may start
// while launch 1 runs (programmatic dependent launch) and waits for it on the
// GPU before it reads lambda; it takes the warp tasks in reverse plan order,
// so the points the forward pass read last, still in L2, come first.
#include <cstring>

#include "lsefit_device.cuh"
#include "lsefit_host.h"

namespace lsefit {

constexpr int kBwBlock = 256;
// Share of its points (1/kBwPrefetchDiv; 0: none) a gradient warp prefetches
// into L2 while the lambda launch runs.
#ifndef LSEFIT_BW_PREFETCH_DIV
#define LSEFIT_BW_PREFETCH_DIV 2
#endif
constexpr int kBwPrefetchDiv = LSEFIT_BW_PREFETCH_DIV;

struct BwParams {
    const void* x;
    const void* y;
    void* dx;
    void* dy;
    const int64_t* offsets;
    const int32_t* degree;
    int64_t num_series;
    int m_max;
    const double* Xt;       // [S][m_max+1]
    const double* map;      // [S][2] or null
    const double* lambda;   // [S][m_max+1] (workspace)
    const float* lamf;      // [S][m_max+1] FP32 copies for the FP32 point pass (workspace)
    const float* xtf;       // [S][m_max+1]
    const float2* mapf;     // [S] (c, s) as FP32
    const int32_t* status;  // [S]
    const int4* block_tasks;
    int n_block_tasks;
    const int4* warp_tasks;  // {series, first point (low, high), length}
    int n_warp_tasks;
    int64_t warp_task_len;  // common length of the warp tasks, 0 when they differ
    unsigned* counters;     // [0] block queue, [1] warp queue, [2] exited blocks
};

// ---------------------------------------------------------------------------
// launch 1: lambda per series
// ---------------------------------------------------------------------------
// Also writes FP32 copies of lambda, Xt and (c, s) so that the point pass of
// FP32 data runs no FP64 instruction (FP64 is 1/64 rate on GB300).
template <int NMAX>
__global__ void lambda_kernel(int64_t S, int m_max, double eps, const int32_t* degree, const double* sums,
                              const double* map, const double* gX, const double* Xt, double* lambda,
                              float* lamf, float* xtf, float2* mapf, int32_t* status, unsigned* counters) {
    griddep_launch_dependents();  // the point pass may start its set-up now
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < 3) counters[s] = 0u;  // the point pass's queue counters (no initialization needed)
    if (s >= S) return;
    const int nc = m_max + 1;
    const int m = degree[s];
    double* lam = lambda + s * nc;
    for (int j = 0; j < nc; ++j) {
        lam[j] = 0.0;
        lamf[s * nc + j] = 0.0f;
        xtf[s * nc + j] = (float)Xt[s * nc + j];
    }
    mapf[s] = map ? make_float2((float)map[2 * s], (float)map[2 * s + 1]) : make_float2(0.0f, 1.0f);
    if (m < 1 || m > m_max || m > NMAX) {
        status[s] = LSEFIT_ERR_INVALID_ARG;
        return;
    }
    const double* Srow = sums + s * (3 * m_max + 2);
    double c = 0.0, sc = 1.0;
    bool ok = true;
    if (map) {
        c = map[2 * s];
        sc = map[2 * s + 1];
        ok = isfinite(c) && isfinite(sc) && sc != 0.0;
    }
    int st = fit_precheck<NMAX>(m, Srow, Srow + 2 * m + 1, ok);
    constexpr int N = NMAX + 1;
    double gt[N], z[N];
    // identity map (c = 0, s = 1): gt = gX, no transform (skipped when every
    // active lane of the warp has it: FP64 instructions cost the warp the same
    // for one lane as for 32)
    const bool ident = c == 0.0 && sc == 1.0;
    if (__all_sync(__activemask(), ident) && st == LSEFIT_OK) {
        const double* g = gX + s * nc;
#pragma unroll
        for (int k = 0; k < N; ++k) gt[k] = k <= m ? g[k] : 0.0;
        bool fin = true;
#pragma unroll
        for (int k = 0; k < N; ++k) fin = fin && finite_bits(gt[k]);
        st = fin ? hankel_ge<NMAX>(m, Srow, gt, z, eps) : LSEFIT_ERR_NONFINITE;
    } else if (st == LSEFIT_OK) {
        // gt_k = sum_{j<=k} C(k,j) s^k (-c)^(k-j) gX_j
        const double* g = gX + s * nc;
        double binom[N];
#pragma unroll
        for (int j = 0; j < N; ++j) binom[j] = 0.0;
        binom[0] = 1.0;
        double sk = 1.0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            gt[k] = 0.0;
            if (k <= m) {
                if (k > 0) {
#pragma unroll
                    for (int j = N - 1; j >= 1; --j) binom[j] += binom[j - 1];
                    sk *= sc;
                }
                double acc = 0.0, cp = 1.0;
#pragma unroll
                for (int j = N - 1; j >= 0; --j) {
                    if (j <= k) {
                        acc = fma(binom[j] * sk * cp, g[j], acc);
                        cp *= -c;
                    }
                }
                gt[k] = acc;
            }
        }
        bool fin = true;
#pragma unroll
        for (int k = 0; k < N; ++k) fin = fin && finite_bits(gt[k]);
        st = fin ? hankel_ge<NMAX>(m, Srow, gt, z, eps) : LSEFIT_ERR_NONFINITE;
    }
    if (st == LSEFIT_OK) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j <= m) {
                lam[j] = z[j];
                lamf[s * nc + j] = (float)z[j];
            }
        }
    }
    status[s] = st;
}

// ---------------------------------------------------------------------------
// launch 2: gradients per point
// ---------------------------------------------------------------------------
template <int DT>
struct OutT {
    typedef float T;
};
template <>
struct OutT<LSEFIT_F64> {
    typedef double T;
};

// Horner's rule with derivative for (lambda, f) on a pair of points.
template <int M>
__device__ __forceinline__ void grad_pair(const u64* lam, const u64* xt, u64 t, u64 y, u64 s2, u64& dxv,
                                          u64& dyv) {
    u64 lv = lam[M], ld = 0ull, fv = xt[M], fd = 0ull;
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        ld = fma2(ld, t, lv);
        lv = fma2(lv, t, lam[j]);
        fd = fma2(fd, t, fv);
        fv = fma2(fv, t, xt[j]);
    }
    const u64 r = sub2(y, fv);
    // s * (ld * r - lv * fd)
    const u64 a = mul2(lv, fd);
    const u64 g = fma2(ld, r, a ^ 0x8000000080000000ull);  // ld*r + (-(lv*fd))
    dxv = mul2(g, s2);
    dyv = lv;
}

template <int M, int DT>
__device__ __forceinline__ void grad_range_f32(const BwParams& p, int64_t b, int64_t e, int64_t rank,
                                               int64_t nthreads, const float* lam32, const float* xt32,
                                               float cf, float sf) {
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec;
    u64 lam[M + 1], xt[M + 1];
#pragma unroll
    for (int j = 0; j <= M; ++j) {
        const float l = lam32[j], f = xt32[j];
        lam[j] = pk2(l, l);
        xt[j] = pk2(f, f);
    }
    const u64 c2 = pk2(cf, cf), s2 = pk2(sf, sf);
    float* dx = static_cast<float*>(p.dx);
    float* dy = static_cast<float*>(p.dy);
    // vector path needs x, y, dx, dy at the same offset within their 16-byte groups
    // (outputs are FP32: for BF16 data the output vectors are 2x wider; scalar path then)
    int64_t head, nvec;
    split_range<DT>(p.x, p.y, b, e, head, nvec);
    const uintptr_t xa = reinterpret_cast<uintptr_t>(p.x) + (uintptr_t)b * ES;
    const uintptr_t da = reinterpret_cast<uintptr_t>(dx) + (uintptr_t)b * 4;
    const uintptr_t ea = reinterpret_cast<uintptr_t>(dy) + (uintptr_t)b * 4;
    if (DT != LSEFIT_F32 || (xa & 15) != (da & 15) || (da & 15) != (ea & 15)) {
        head = e - b;
        nvec = 0;
    }
    const uint4* xv = reinterpret_cast<const uint4*>(static_cast<const char*>(p.x) + (b + head) * ES);
    const uint4* yv = reinterpret_cast<const uint4*>(static_cast<const char*>(p.y) + (b + head) * ES);
    float4* dxv = reinterpret_cast<float4*>(dx + b + head);
    float4* dyv = reinterpret_cast<float4*>(dy + b + head);
    // one 16-byte vector of x and y -> 4 gradients of each
    auto grad_vec = [&](uint4 xr, uint4 yr, float4& ox, float4& oy) {
        u64 ta = mul2(sub2(pk2(__uint_as_float(xr.x), __uint_as_float(xr.y)), c2), s2);
        u64 tb = mul2(sub2(pk2(__uint_as_float(xr.z), __uint_as_float(xr.w)), c2), s2);
        u64 ya = pk2(__uint_as_float(yr.x), __uint_as_float(yr.y));
        u64 yb = pk2(__uint_as_float(yr.z), __uint_as_float(yr.w));
        u64 gxa, gya, gxb, gyb;
        grad_pair<M>(lam, xt, ta, ya, s2, gxa, gya);
        grad_pair<M>(lam, xt, tb, yb, s2, gxb, gyb);
        up2(gxa, ox.x, ox.y);
        up2(gxb, ox.z, ox.w);
        up2(gya, oy.x, oy.y);
        up2(gyb, oy.z, oy.w);
    };
    constexpr int U = 4;  // vectors in flight per thread
    int64_t v = rank;
    for (; v + (U - 1) * nthreads < nvec; v += U * nthreads) {
        uint4 xr[U], yr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xr[u] = ld_stream16(xv + v + u * nthreads);
            yr[u] = ld_stream16(yv + v + u * nthreads);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float4 ox, oy;
            grad_vec(xr[u], yr[u], ox, oy);
            __stcs(dxv + v + u * nthreads, ox);
            __stcs(dyv + v + u * nthreads, oy);
        }
    }
    for (; v < nvec; v += nthreads) {
        float4 ox, oy;
        grad_vec(ld_stream16(xv + v), ld_stream16(yv + v), ox, oy);
        __stcs(dxv + v, ox);
        __stcs(dyv + v, oy);
    }
    const int64_t tail0 = b + head + nvec * PV;
    const int64_t nscalar = head + (e - tail0);
    for (int64_t q = rank; q < nscalar; q += nthreads) {
        const int64_t i = q < head ? b + q : tail0 + (q - head);
        const float xs = Elem<DT>::ld(p.x, i), ys = Elem<DT>::ld(p.y, i);
        const float ts = __fmul_rn(__fsub_rn(xs, cf), sf);
        u64 gx, gy;
        grad_pair<M>(lam, xt, pk2(ts, 0.0f), pk2(ys, 0.0f), s2, gx, gy);
        float a0, a1, b0, b1;
        up2(gx, a0, a1);
        up2(gy, b0, b1);
        dx[i] = a0;
        dy[i] = b0;
    }
}

template <int M>
__device__ __forceinline__ void grad_range_f64(const BwParams& p, int64_t b, int64_t e, int64_t rank,
                                               int64_t nthreads, const double* lam, const double* xt,
                                               double c, double sc) {
    double* dx = static_cast<double*>(p.dx);
    double* dy = static_cast<double*>(p.dy);
    for (int64_t i = b + rank; i < e; i += nthreads) {
        const double t = sc * (Elem<LSEFIT_F64>::ld64(p.x, i) - c);
        double lv = lam[M], ld = 0.0, fv = xt[M], fd = 0.0;
#pragma unroll
        for (int j = M - 1; j >= 0; --j) {
            ld = fma(ld, t, lv);
            lv = fma(lv, t, lam[j]);
            fd = fma(fd, t, fv);
            fv = fma(fv, t, xt[j]);
        }
        const double r = Elem<LSEFIT_F64>::ld64(p.y, i) - fv;
        dx[i] = sc * (ld * r - lv * fd);
        dy[i] = lv;
    }
}

// Zero gradients of a series that has no valid adjoint.
template <int DT>
__device__ __forceinline__ void zero_range(const BwParams& p, int64_t b, int64_t e, int64_t rank, int64_t nthreads) {
    typedef typename OutT<DT>::T T;
    T* dx = static_cast<T*>(p.dx);
    T* dy = static_cast<T*>(p.dy);
    for (int64_t i = b + rank; i < e; i += nthreads) {
        dx[i] = (T)0;
        dy[i] = (T)0;
    }
}

template <int DT, int M>
__device__ __forceinline__ void grad_task(const BwParams& p, int64_t s, int64_t b, int64_t e, int64_t rank,
                                          int64_t nthreads) {
    const int nc = p.m_max + 1;
    if constexpr (DT == LSEFIT_F64) {
        const double* lam = p.lambda + s * nc;
        const double* xt = p.Xt + s * nc;
        const double c = p.map ? p.map[2 * s] : 0.0;
        const double sc = p.map ? p.map[2 * s + 1] : 1.0;
        double l[M + 1], f[M + 1];
#pragma unroll
        for (int j = 0; j <= M; ++j) {
            l[j] = lam[j];
            f[j] = xt[j];
        }
        grad_range_f64<M>(p, b, e, rank, nthreads, l, f, c, sc);
    } else {
        const float2 cs = p.mapf[s];
        grad_range_f32<M, DT>(p, b, e, rank, nthreads, p.lamf + s * nc, p.xtf + s * nc, cs.x, cs.y);
    }
}

template <int DT>
__device__ __forceinline__ void grad_dispatch(const BwParams& p, int64_t s, int64_t b, int64_t e, int64_t rank,
                                              int64_t nthreads) {
    const int m = p.degree[s];
    if (p.status[s] != LSEFIT_OK || m < 1 || m > p.m_max) {
        zero_range<DT>(p, b, e, rank, nthreads);
        return;
    }
    switch (m) {
        case 1: grad_task<DT, 1>(p, s, b, e, rank, nthreads); break;
        case 2: grad_task<DT, 2>(p, s, b, e, rank, nthreads); break;
        case 3: grad_task<DT, 3>(p, s, b, e, rank, nthreads); break;
        case 4: grad_task<DT, 4>(p, s, b, e, rank, nthreads); break;
        case 5: grad_task<DT, 5>(p, s, b, e, rank, nthreads); break;
        case 6: grad_task<DT, 6>(p, s, b, e, rank, nthreads); break;
        case 7: grad_task<DT, 7>(p, s, b, e, rank, nthreads); break;
        default: grad_task<DT, 8>(p, s, b, e, rank, nthreads); break;
    }
}

template <int DT>
__global__ void __launch_bounds__(kBwBlock) grad_kernel(__grid_constant__ const BwParams p) {
    __shared__ int s_task;
    const int tid = threadIdx.x, lane = tid & 31;
    // Tasks of one common length are split evenly by points over all warps
    // (numbered warp-major, so every SM gets the same share): warp wid takes
    // [wid * per, +per) of the points in reverse plan order.
    const int64_t L = p.warp_task_len;
    const int64_t total = (int64_t)p.n_warp_tasks * L;
    const int64_t nw = (int64_t)gridDim.x * (kBwBlock / 32);
    const int64_t wid = (int64_t)(tid >> 5) * gridDim.x + blockIdx.x;
    const int64_t per = L > 0 ? ((total + nw - 1) / nw + 3) / 4 * 4 : 0;  // whole 16-byte vectors of FP32 points
    if (kBwPrefetchDiv > 0 && L > 0 && p.n_block_tasks == 0) {
        // While the lambda launch solves, DRAM is idle: bring the first part of
        // this warp's points into L2 (the reads do not depend on lambda).
        constexpr int ES = Elem<DT>::kSize, LINE = 128 / ES;  // points per 128-byte line
        int64_t pos = min(total, wid * per);
        const int64_t hi = min(total, pos + per / (kBwPrefetchDiv > 0 ? kBwPrefetchDiv : 1));
        while (pos < hi) {
            const int64_t r = pos / L;
            const int64_t seg = min(hi, (r + 1) * L);
            const int4 task = p.warp_tasks[p.n_warp_tasks - 1 - r];
            const int64_t first = ((int64_t)(unsigned)task.z << 32) | (unsigned)task.y;
            for (int64_t q = pos + (int64_t)lane * LINE; q < seg; q += 32 * LINE) {
                prefetch_l2(static_cast<const char*>(p.x) + (first + (q - r * L)) * ES);
                prefetch_l2(static_cast<const char*>(p.y) + (first + (q - r * L)) * ES);
            }
            pos = seg;
        }
    }
    // lambda, the FP32 copies and the queue counters come from the lambda launch
    griddep_wait();
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(&p.counters[0], 1u);
        __syncthreads();
        const int t = s_task;
        __syncthreads();
        if (t >= p.n_block_tasks) break;
        const int4 task = p.block_tasks[t];
        const int64_t s = task.x;
        const int64_t b0 = p.offsets[s], e0 = p.offsets[s + 1];
        const int64_t per = ((e0 - b0 + task.z - 1) / task.z + 7) / 8 * 8;
        const int64_t b = min(b0 + (int64_t)task.y * per, e0);
        const int64_t e = min(b + per, e0);
        grad_dispatch<DT>(p, s, b, e, tid, kBwBlock);
    }
    // warp tasks in reverse plan order: the forward pass read the last tasks of
    // the plan last, so their points are the ones still held in L2.  The even
    // split balances a batch of fewer tasks than twice the warps; tasks of
    // different lengths are drawn whole.
    if (L > 0) {
        int64_t pos = min(total, wid * per);
        const int64_t hi = min(total, pos + per);
        while (pos < hi) {
            const int64_t r = pos / L;                 // r-th task from the end of the plan
            const int64_t seg = min(hi, (r + 1) * L);  // this task's part of the range
            const int4 task = p.warp_tasks[p.n_warp_tasks - 1 - r];
            const int64_t first = ((int64_t)(unsigned)task.z << 32) | (unsigned)task.y;
            grad_dispatch<DT>(p, task.x, first + (pos - r * L), first + (seg - r * L), lane, 32);
            pos = seg;
        }
    } else
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&p.counters[1], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= p.n_warp_tasks) break;
        const int64_t s = p.warp_tasks[p.n_warp_tasks - 1 - t].x;
        grad_dispatch<DT>(p, s, p.offsets[s], p.offsets[s + 1], lane, 32);
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

}  // namespace lsefit

using namespace lsefit;

// Workspace: counters | lambda [S][m_max+1] FP64 | lambda, Xt [S][m_max+1] FP32 | (c, s) [S] FP32.
static size_t bw_off_lamf(const lsefit_plan* plan) {
    return kAlign + align_up((size_t)plan->num_series * (plan->m_max + 1) * sizeof(double), kAlign);
}
static size_t bw_off_xtf(const lsefit_plan* plan) {
    return bw_off_lamf(plan) + align_up((size_t)plan->num_series * (plan->m_max + 1) * sizeof(float), kAlign);
}
static size_t bw_off_mapf(const lsefit_plan* plan) {
    return bw_off_xtf(plan) + align_up((size_t)plan->num_series * (plan->m_max + 1) * sizeof(float), kAlign);
}

extern "C" size_t lsefit_backward_workspace_size(const lsefit_plan* plan) {
    if (plan == nullptr || plan->m_max < 1 || plan->num_series < 0) return 0;
    return bw_off_mapf(plan) + align_up((size_t)plan->num_series * sizeof(float2), kAlign);
}

extern "C" int lsefit_backward(const lsefit_batch* batch, const lsefit_plan* plan, const double* sums,
                               const double* Xt, const double* map, const double* gX, void* dx, void* dy,
                               int32_t* status, void* workspace, size_t workspace_bytes,
                               lsefit_stream_t stream) {
    if (batch == nullptr || plan == nullptr || status == nullptr) return LSEFIT_ERR_INVALID_ARG;
    const lsefit_batch& b = *batch;
    if (b.num_series != plan->num_series || b.m_max != plan->m_max || b.m_max < 1 ||
        b.m_max > LSEFIT_MAX_DEGREE)
        return LSEFIT_ERR_INVALID_ARG;
    if (b.dtype < LSEFIT_F64 || b.dtype > LSEFIT_BF16) return LSEFIT_ERR_INVALID_ARG;
    if (b.basis != LSEFIT_BASIS_MONOMIAL) return LSEFIT_ERR_UNSUPPORTED;  // evaluates t^k polynomials
    if (b.accum < LSEFIT_ACCUM_NAIVE || b.accum > LSEFIT_ACCUM_F64) return LSEFIT_ERR_INVALID_ARG;
    if (b.num_series == 0) return LSEFIT_OK;
    if (sums == nullptr || Xt == nullptr || gX == nullptr || b.offsets == nullptr || b.degree == nullptr)
        return LSEFIT_ERR_INVALID_ARG;
    if (plan->total_points > 0 && (b.x == nullptr || b.y == nullptr || dx == nullptr || dy == nullptr))
        return LSEFIT_ERR_INVALID_ARG;
    if (workspace == nullptr || !aligned(workspace, kAlign) ||
        workspace_bytes < lsefit_backward_workspace_size(plan))
        return LSEFIT_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    double* lambda = reinterpret_cast<double*>(ws + kAlign);
    float* lamf = reinterpret_cast<float*>(ws + bw_off_lamf(plan));
    float* xtf = reinterpret_cast<float*>(ws + bw_off_xtf(plan));
    float2* mapf = reinterpret_cast<float2*>(ws + bw_off_mapf(plan));
    // one warp per block, so the solves (FP64-bound: an FP64 instruction costs a
    // warp the same for one lane as for 32) spread over as many SMs as possible
    const int threads = 32;
    const int64_t blocks = (b.num_series + threads - 1) / threads;
    auto lk = b.m_max <= 3 ? lambda_kernel<3> : b.m_max <= 5 ? lambda_kernel<5> : lambda_kernel<8>;
    lk<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(b.num_series, b.m_max, singular_eps(b.accum),
                                                              b.degree, sums, map, gX, Xt, lambda, lamf, xtf,
                                                              mapf, status, reinterpret_cast<unsigned*>(ws));
    if (cudaGetLastError() != cudaSuccess) return LSEFIT_ERR_CUDA;

    BwParams p;
    p.x = b.x;
    p.y = b.y;
    p.dx = dx;
    p.dy = dy;
    p.offsets = b.offsets;
    p.degree = b.degree;
    p.num_series = b.num_series;
    p.m_max = b.m_max;
    p.Xt = Xt;
    p.map = map;
    p.lambda = lambda;
    p.lamf = lamf;
    p.xtf = xtf;
    p.mapf = mapf;
    p.status = status;
    p.block_tasks = reinterpret_cast<const int4*>(plan->block_tasks);
    p.n_block_tasks = plan->n_block_tasks;
    p.warp_tasks = reinterpret_cast<const int4*>(plan->warp_tasks);
    p.n_warp_tasks = plan->n_warp_tasks;
    p.warp_task_len = plan->warp_task_len;
    p.counters = reinterpret_cast<unsigned*>(ws);
    auto gk = b.dtype == LSEFIT_F64 ? grad_kernel<LSEFIT_F64>
              : b.dtype == LSEFIT_F32 ? grad_kernel<LSEFIT_F32> : grad_kernel<LSEFIT_BF16>;
    int dev = 0;
    const int sms = current_sm_count(&dev);
    if (sms <= 0) return LSEFIT_ERR_CUDA;
    const int occ = occupancy_blocks(reinterpret_cast<const void*>(gk), kBwBlock, 0);
    int64_t grid = (int64_t)sms * occ;
    const int64_t useful = (int64_t)plan->n_block_tasks + (plan->n_warp_tasks + 7) / 8;
    if (useful < grid) grid = useful;
    if (grid < 1) grid = 1;
    // the point pass starts while the lambda solves run and waits for them on the GPU
    if (launch_after_prior(gk, dim3((unsigned)grid), dim3(kBwBlock), 0, (cudaStream_t)stream, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return LSEFIT_ERR_CUDA;
    }
    return LSEFIT_OK;
}
