// lsefit_range.cu -- interval prepass: per-series [min x, max x], for fits
// whose caller does not know the interval of the affine map.
//
// Not in the paper.  The map t = s (x - c) with c = (lo+hi)/2, s = 2/(hi-lo)
// keeps the Hankel system of Section II well-conditioned; when lo and hi are
// not given they are the extremes of the series' own abscissae.  Minimum and
// maximum are exact and independent of the order of evaluation, so blocks
// combine with atomic maxima on order-preserving integer encodings: the
// maximum as enc(x), the minimum as ~enc(x), both with 0 as the neutral
// value.  A second launch decodes the intervals and zeroes the slots again.
#include "lsefit_device.cuh"
#include "lsefit_host.h"

namespace lsefit {

constexpr int kRgBlock = 256;

// Monotone map of a double onto unsigned 64-bit integers (a < b <=> enc(a) < enc(b)).
__device__ __forceinline__ unsigned long long enc64(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dec64(unsigned long long e) {
    const unsigned long long u = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    return __longlong_as_double((long long)u);
}

struct RgParams {
    const void* x;
    const int64_t* offsets;
    const int4* block_tasks;
    int n_block_tasks;
    const int4* warp_tasks;
    int n_warp_tasks;
    unsigned long long* slots;  // [num_series][2]: enc(max), ~enc(min); zero between calls
    unsigned* counters;         // [0] block queue, [1] warp queue, [2] exited blocks
};

template <int DT>
__device__ __forceinline__ void range_of(const void* x, int64_t b, int64_t e, int64_t rank, int64_t nthreads,
                                         double& lo, double& hi) {
    for (int64_t i = b + rank; i < e; i += nthreads) {
        const double v = Elem<DT>::ld64(x, i);
        if (v == v) {  // NaN never lowers or raises the range
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
    }
}

// One pass over a task's points in FP32 for FP32/BF16 data (exact: FP32 and
// BF16 values compare the same way as their FP64 promotions).
template <int DT>
__device__ __forceinline__ void range_of_f32(const void* x, int64_t b, int64_t e, int64_t rank,
                                             int64_t nthreads, float& lo, float& hi) {
    for (int64_t i = b + rank; i < e; i += nthreads) {
        const float v = Elem<DT>::ld(x, i);
        lo = fminf(lo, v);  // fminf/fmaxf ignore a NaN operand
        hi = fmaxf(hi, v);
    }
}

template <int DT>
__global__ void __launch_bounds__(kRgBlock) range_kernel(__grid_constant__ const RgParams p) {
    __shared__ int s_task;
    const int tid = threadIdx.x, lane = tid & 31;
    // one series range contributes through lane 0's atomics after a warp reduction
    auto publish = [&](int64_t s, float lo32, float hi32, double lo64, double hi64, bool f64) {
        double lo = f64 ? lo64 : (double)lo32, hi = f64 ? hi64 : (double)hi32;
        if (!(lo <= hi)) return;  // nothing seen
        atomicMax(&p.slots[2 * s], enc64(hi));
        atomicMax(&p.slots[2 * s + 1], ~enc64(lo));
    };
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(&p.counters[0], 1u);
        __syncthreads();
        const int t = s_task;
        __syncthreads();
        if (t >= p.n_block_tasks) break;
        const int4 task = p.block_tasks[t];
        const int64_t s = task.x, b0 = p.offsets[s], e0 = p.offsets[s + 1];
        const int64_t per = ((e0 - b0 + task.z - 1) / task.z + 7) / 8 * 8;
        const int64_t b = min(b0 + (int64_t)task.y * per, e0), e = min(b + per, e0);
        if constexpr (DT == LSEFIT_F64) {
            double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
            range_of<DT>(p.x, b, e, tid, kRgBlock, lo, hi);
            for (int o = 16; o > 0; o >>= 1) {
                lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) publish(s, 0.f, 0.f, lo, hi, true);
        } else {
            float lo = __int_as_float(0x7f800000), hi = -lo;
            range_of_f32<DT>(p.x, b, e, tid, kRgBlock, lo, hi);
            for (int o = 16; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) publish(s, lo, hi, 0.0, 0.0, false);
        }
    }
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&p.counters[1], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= p.n_warp_tasks) break;
        const int4 task = p.warp_tasks[t];
        const int64_t s = task.x, b = p.offsets[s], e = p.offsets[s + 1];
        if constexpr (DT == LSEFIT_F64) {
            double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
            range_of<DT>(p.x, b, e, lane, 32, lo, hi);
            for (int o = 16; o > 0; o >>= 1) {
                lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) publish(s, 0.f, 0.f, lo, hi, true);
        } else {
            float lo = __int_as_float(0x7f800000), hi = -lo;
            range_of_f32<DT>(p.x, b, e, lane, 32, lo, hi);
            for (int o = 16; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) publish(s, lo, hi, 0.0, 0.0, false);
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

// Decode the slots into [lo, hi] (NaN for a series with no finite point) and
// zero them for the next call.
__global__ void range_finish_kernel(int64_t S, unsigned long long* slots, double* interval) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const unsigned long long emax = slots[2 * s], nmin = slots[2 * s + 1];
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    if (emax == 0ull) {
        interval[2 * s] = qnan;
        interval[2 * s + 1] = qnan;
    } else {
        interval[2 * s] = dec64(~nmin);
        interval[2 * s + 1] = dec64(emax);
    }
    slots[2 * s] = 0ull;
    slots[2 * s + 1] = 0ull;
}

}  // namespace lsefit

using namespace lsefit;

extern "C" size_t lsefit_range_workspace_size(const lsefit_plan* plan) {
    if (plan == nullptr || plan->num_series < 0) return 0;
    return kAlign + align_up((size_t)plan->num_series * 16, kAlign);
}

extern "C" int lsefit_range(const lsefit_batch* batch, const lsefit_plan* plan, double* interval,
                            void* workspace, size_t workspace_bytes, lsefit_stream_t stream) {
    if (batch == nullptr || plan == nullptr || interval == nullptr) return LSEFIT_ERR_INVALID_ARG;
    const lsefit_batch& b = *batch;
    if (b.num_series != plan->num_series) return LSEFIT_ERR_INVALID_ARG;
    if (b.dtype < LSEFIT_F64 || b.dtype > LSEFIT_BF16) return LSEFIT_ERR_INVALID_ARG;
    if (b.num_series == 0) return LSEFIT_OK;
    if (b.offsets == nullptr || (plan->total_points > 0 && b.x == nullptr)) return LSEFIT_ERR_INVALID_ARG;
    if ((plan->n_block_tasks > 0 && plan->block_tasks == nullptr) ||
        (plan->n_warp_tasks > 0 && plan->warp_tasks == nullptr))
        return LSEFIT_ERR_INVALID_ARG;
    if (workspace == nullptr || !aligned(workspace, kAlign) ||
        workspace_bytes < lsefit_range_workspace_size(plan))
        return LSEFIT_ERR_WORKSPACE;
    RgParams p;
    p.x = b.x;
    p.offsets = b.offsets;
    p.block_tasks = reinterpret_cast<const int4*>(plan->block_tasks);
    p.n_block_tasks = plan->n_block_tasks;
    p.warp_tasks = reinterpret_cast<const int4*>(plan->warp_tasks);
    p.n_warp_tasks = plan->n_warp_tasks;
    p.counters = static_cast<unsigned*>(workspace);
    p.slots = reinterpret_cast<unsigned long long*>(static_cast<char*>(workspace) + kAlign);
    auto k = b.dtype == LSEFIT_F64 ? range_kernel<LSEFIT_F64>
             : b.dtype == LSEFIT_F32 ? range_kernel<LSEFIT_F32> : range_kernel<LSEFIT_BF16>;
    int dev = 0;
    const int sms = current_sm_count(&dev);
    if (sms <= 0) return LSEFIT_ERR_CUDA;
    const int occ = occupancy_blocks(reinterpret_cast<const void*>(k), kRgBlock, 0);
    int64_t grid = (int64_t)sms * occ;
    const int64_t useful = (int64_t)plan->n_block_tasks + (plan->n_warp_tasks + 7) / 8;
    if (useful < grid) grid = useful;
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, kRgBlock, 0, (cudaStream_t)stream>>>(p);
    if (cudaGetLastError() != cudaSuccess) return LSEFIT_ERR_CUDA;
    const int64_t fb = (b.num_series + 255) / 256;
    range_finish_kernel<<<(unsigned)fb, 256, 0, (cudaStream_t)stream>>>(b.num_series, p.slots, interval);
    return cudaGetLastError() == cudaSuccess ? LSEFIT_OK : LSEFIT_ERR_CUDA;
}
