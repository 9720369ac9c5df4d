// lsefit_powersums.cu -- single-series streaming pass (Section II: the
// entries of A and B are the sums S_k = sum_i x_i^k and T_k = sum_i x_i^k y_i).
//
// One grid-stride pass over the points.  Each thread reads 16-byte vectors of
// x and y (UNROLL of each in flight), maps them (t = s (x - c)), builds the
// powers t^k by a running product and adds them into 3m+1 accumulators, two
// points per packed-FP32 instruction.  The block then reduces its threads'
// accumulators exactly to double-float, converts the block totals to FP64
// and stores them as per-block partials; the last block to finish (ticket
// counter, no waiting) adds the partials in FP64 in a fixed order and writes
// S_0..S_2m, T_0..T_m.  The result depends only on n and the launch shape.
#include <mutex>

#include "lsefit_device.cuh"
#include "lsefit_host.h"

namespace lsefit {

constexpr int kPSBlock = 256;

struct PSParams {
    const void* x;
    const void* y;
    int64_t n;
    const double* interval;
    double* sums;
    double* map_out;
    int32_t* status;
    double* partials;       // [gridDim.x][3m+1]
    unsigned int* ticket;   // zero between calls
    // fused solve (lsefit_fit): degrees m_lo..m, one per lane of warp 0
    int m_lo;
    double eps;             // singularity threshold epsilon of the accumulation
    double* X;              // [m-m_lo+1][m+1] or null (no solve)
    double* Xt;             // same shape or null
    int32_t* fit_status;    // [m-m_lo+1]
};

// The fused solves of lsefit_fit, kept out of line so that their FP64
// register demand does not reshape the streaming loop of the kernel.
template <int M>
__device__ __noinline__ void ps_solve_degrees(const PSParams& p, const double* tot, double c, double s,
                                              bool map_ok, int lane) {
    const int d = p.m_lo + lane;
    const int st = solve_hankel_rt<M>(d, tot, tot + 2 * M + 1, c, s, map_ok, p.eps,
                                      p.Xt ? p.Xt + lane * (M + 1) : nullptr, p.X + lane * (M + 1), M + 1);
    p.fit_status[lane] = st;
}

// Last block: fixed-order FP64 sum of the per-block partials, then the outputs.
template <int M>
__device__ void ps_finish(const PSParams& p, bool map_ok, double c, double s, double* comb) {
    constexpr int N = 3 * M + 1;
    constexpr int J = kPSBlock / N;
    __shared__ double tot_s[N + 1];
    const int tid = threadIdx.x;
    const int G = gridDim.x;
    if (tid < N * J) {
        const int a = tid / J, j = tid % J;
        double v = 0.0;
        for (int b = j; b < G; b += J) v += __ldcg(p.partials + (size_t)b * N + a);
        comb[tid] = v;
    }
    __syncthreads();
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    if (tid < N) {
        double tot = 0.0;
        for (int j = 0; j < J; ++j) tot += comb[tid * J + j];
        // accumulator a holds S_{a+1} (a < 2M) or T_{a-2M}; in the output
        // layout S_0..S_2M, T_0..T_M both land at index a + 1.
        tot_s[tid + 1] = map_ok ? tot : qnan;
        if (p.sums) p.sums[tid + 1] = map_ok ? tot : qnan;
    }
    if (tid == 0) {
        tot_s[0] = map_ok ? (double)p.n : qnan;
        if (p.sums) p.sums[0] = map_ok ? (double)p.n : qnan;
        if (p.map_out) {
            p.map_out[0] = map_ok ? c : qnan;
            p.map_out[1] = map_ok ? s : qnan;
        }
        if (p.status) p.status[0] = map_ok ? LSEFIT_OK : LSEFIT_ERR_BAD_INTERVAL;
        *p.ticket = 0u;  // ready for the next call
    }
    if (p.X != nullptr) {
        // every requested degree d = m_lo + lane solves from the prefix of the
        // degree-M sums (S_0..S_2d, T_0..T_d), all lanes in step
        __syncthreads();
        const int lane = tid;
        if (tid < 32 && lane <= M - p.m_lo) ps_solve_degrees<M>(p, tot_s, c, s, map_ok, lane);
    }
}

// Shared tail of both kernels: store the block partial, take a ticket, and
// let the last block combine.
template <int M>
__device__ __forceinline__ void ps_publish(const PSParams& p, const double* blk, bool map_ok,
                                           double c, double s, double* comb) {
    constexpr int N = 3 * M + 1;
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    if (tid < N) {
        p.partials[(size_t)blockIdx.x * N + tid] = blk[tid];
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(p.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ps_finish<M>(p, map_ok, c, s, comb);
}

// FP32 / BF16 storage, NAIVE or COMP accumulation.
template <int M, int DT, bool COMP, bool MAP, int UNROLL>
__global__ void __launch_bounds__(kPSBlock, pass_min_blocks<M>()) ps_kernel_f32(__grid_constant__ const PSParams p) {
    constexpr int N = 3 * M + 1;
    __shared__ dflt red[(kPSBlock / 32) * kPSBlock];
    __shared__ double blk[N];
    __shared__ double comb[kPSBlock];

    double cd, sd;
    const bool map_ok = map_constants(MAP ? p.interval : nullptr, true, cd, sd);
    AccF32<M, COMP> A;
    A.init();
    const int64_t nthr = (int64_t)gridDim.x * kPSBlock;
    const int64_t gtid = (int64_t)blockIdx.x * kPSBlock + threadIdx.x;
    accumulate_range<M, DT, COMP, MAP, UNROLL>(A, p.x, p.y, 0, p.n, gtid, nthr, (float)cd, (float)sd);
    block_reduce_df<kPSBlock, N>([&](int a) { return A.result(a); }, red, blk);
    ps_publish<M>(p, blk, map_ok, cd, sd, comb);
}

// FP64 accumulation (any storage): map, powers and sums in FP64.
template <int M, int DT, bool MAP, int UNROLL>
__global__ void __launch_bounds__(kPSBlock) ps_kernel_f64(__grid_constant__ const PSParams p) {
    constexpr int N = 3 * M + 1;
    __shared__ double red[(kPSBlock / 32) * kPSBlock];
    __shared__ double blk[N];
    __shared__ double comb[kPSBlock];

    double c, s;
    const bool map_ok = map_constants(MAP ? p.interval : nullptr, false, c, s);
    AccF64<M> A;
    A.init();
    const int64_t nthr = (int64_t)gridDim.x * kPSBlock;
    const int64_t gtid = (int64_t)blockIdx.x * kPSBlock + threadIdx.x;
    accumulate_range_f64<M, DT, UNROLL, MAP>(A, p.x, p.y, 0, p.n, gtid, nthr, c, s);
    block_reduce_d<kPSBlock, N>([&](int a) { return A.acc[a]; }, red, blk);
    ps_publish<M>(p, blk, map_ok, c, s, comb);
}

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------
typedef void (*ps_kernel_t)(PSParams);

template <int M>
static ps_kernel_t pick_kernel_m(int dtype, int accum, bool map) {
    if (accum == LSEFIT_ACCUM_F64) {
        if (dtype == LSEFIT_F64) return map ? ps_kernel_f64<M, LSEFIT_F64, true, 2> : ps_kernel_f64<M, LSEFIT_F64, false, 2>;
        if (dtype == LSEFIT_F32) return map ? ps_kernel_f64<M, LSEFIT_F32, true, 2> : ps_kernel_f64<M, LSEFIT_F32, false, 2>;
        return map ? ps_kernel_f64<M, LSEFIT_BF16, true, 1> : ps_kernel_f64<M, LSEFIT_BF16, false, 1>;
    }
    const bool comp = accum == LSEFIT_ACCUM_COMP;
    constexpr int UF = M <= 4 ? 4 : 2;  // FP32 vectors in flight per thread
    constexpr int UB = 2;
    if (dtype == LSEFIT_F32) {
        if (comp) return map ? ps_kernel_f32<M, LSEFIT_F32, true, true, UF> : ps_kernel_f32<M, LSEFIT_F32, true, false, UF>;
        return map ? ps_kernel_f32<M, LSEFIT_F32, false, true, UF> : ps_kernel_f32<M, LSEFIT_F32, false, false, UF>;
    }
    if (comp) return map ? ps_kernel_f32<M, LSEFIT_BF16, true, true, UB> : ps_kernel_f32<M, LSEFIT_BF16, true, false, UB>;
    return map ? ps_kernel_f32<M, LSEFIT_BF16, false, true, UB> : ps_kernel_f32<M, LSEFIT_BF16, false, false, UB>;
}

static ps_kernel_t pick_kernel(int m, int dtype, int accum, bool map) {
    switch (m) {
        case 1: return pick_kernel_m<1>(dtype, accum, map);
        case 2: return pick_kernel_m<2>(dtype, accum, map);
        case 3: return pick_kernel_m<3>(dtype, accum, map);
        case 4: return pick_kernel_m<4>(dtype, accum, map);
        case 5: return pick_kernel_m<5>(dtype, accum, map);
        case 6: return pick_kernel_m<6>(dtype, accum, map);
        case 7: return pick_kernel_m<7>(dtype, accum, map);
        default: return pick_kernel_m<8>(dtype, accum, map);
    }
}

}  // namespace lsefit

using namespace lsefit;

extern "C" size_t lsefit_powersums_workspace_size(int m) {
    if (m < 1 || m > LSEFIT_MAX_DEGREE) return 0;
    return kAlign + align_up((size_t)kMaxGrid * (3 * m + 1) * sizeof(double), kAlign);
}

static int launch_powersums(const void* x, const void* y, int64_t n, int dtype, int m, int accum,
                            const double* interval, double* sums, double* map, int32_t* status,
                            void* workspace, size_t workspace_bytes, lsefit_stream_t stream, int m_lo,
                            double* X, double* Xt, int32_t* fit_status) {
    if (m < 1 || m > LSEFIT_MAX_DEGREE || n < 0) return LSEFIT_ERR_INVALID_ARG;
    if (sums == nullptr && X == nullptr) return LSEFIT_ERR_INVALID_ARG;
    if (X != nullptr && (m_lo < 1 || m_lo > m || fit_status == nullptr)) return LSEFIT_ERR_INVALID_ARG;
    if (dtype < LSEFIT_F64 || dtype > LSEFIT_BF16) return LSEFIT_ERR_INVALID_ARG;
    if (accum < LSEFIT_ACCUM_NAIVE || accum > LSEFIT_ACCUM_F64) return LSEFIT_ERR_INVALID_ARG;
    if (dtype == LSEFIT_F64 && accum != LSEFIT_ACCUM_F64) return LSEFIT_ERR_UNSUPPORTED;
    if (n > 0 && (x == nullptr || y == nullptr)) return LSEFIT_ERR_INVALID_ARG;
    if (n >= (int64_t(1) << 53)) return LSEFIT_ERR_INVALID_ARG;  // S_0 must be exact in FP64
    if (workspace == nullptr || !aligned(workspace, kAlign)) return LSEFIT_ERR_WORKSPACE;
    if (workspace_bytes < lsefit_powersums_workspace_size(m)) return LSEFIT_ERR_WORKSPACE;

    if (n > 0) {
        if (resolve_device_pointer(x) != LSEFIT_OK || resolve_device_pointer(y) != LSEFIT_OK) return LSEFIT_ERR_INVALID_ARG;
    }
    const int es = elem_size(dtype);
    const int per_vec = 16 / es;
    PSParams p;
    p.x = x;
    p.y = y;
    p.n = n;
    p.interval = interval;
    p.sums = sums;
    p.map_out = map;
    p.status = status;
    p.ticket = static_cast<unsigned int*>(workspace);
    p.partials = reinterpret_cast<double*>(static_cast<char*>(workspace) + kAlign);
    p.m_lo = m_lo;
    p.eps = singular_eps(accum);
    p.X = X;
    p.Xt = Xt;
    p.fit_status = fit_status;

    ps_kernel_t k = pick_kernel(m, dtype, accum, interval != nullptr);
    int dev = 0;
    const int sms = current_sm_count(&dev);
    if (sms <= 0) return LSEFIT_ERR_CUDA;
    const int occ = occupancy_blocks(reinterpret_cast<const void*>(k), kPSBlock, 0);
    // enough blocks to fill the GPU, but at least ~2 vectors per thread
    const int64_t work = (n + per_vec - 1) / per_vec;
    int64_t want = (work + 2 * kPSBlock - 1) / (2 * kPSBlock);
    int64_t grid = (int64_t)sms * occ;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    if (grid > kMaxGrid) grid = kMaxGrid;
    k<<<(unsigned)grid, kPSBlock, 0, (cudaStream_t)stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? LSEFIT_OK : LSEFIT_ERR_CUDA;
}

extern "C" int lsefit_powersums(const void* x, const void* y, int64_t n, int dtype, int m, int accum,
                                const double* interval, double* sums, double* map, int32_t* status,
                                void* workspace, size_t workspace_bytes, lsefit_stream_t stream) {
    if (sums == nullptr) return LSEFIT_ERR_INVALID_ARG;
    return launch_powersums(x, y, n, dtype, m, accum, interval, sums, map, status, workspace, workspace_bytes,
                            stream, 0, nullptr, nullptr, nullptr);
}

extern "C" int lsefit_fit(const void* x, const void* y, int64_t n, int dtype, int m, int m_lo, int accum,
                          const double* interval, double* X, double* Xt, double* sums, double* map,
                          int32_t* status, void* workspace, size_t workspace_bytes, lsefit_stream_t stream) {
    if (X == nullptr || status == nullptr) return LSEFIT_ERR_INVALID_ARG;
    return launch_powersums(x, y, n, dtype, m, accum, interval, sums, map, nullptr, workspace, workspace_bytes,
                            stream, m_lo, X, Xt, status);
}

// ---------------------------------------------------------------------------
// Allocation-free single-series fit.
//
// Some callers cannot allocate device memory at the time they fit: a service
// that runs under a fixed device-memory budget and forbids allocation after
// start-up, or a plugin host that hands its plugins only input and output
// buffers and offers no allocator.  For them lsefit_fit_noalloc keeps the
// reduction's scratch (the ticket word and the per-block FP64 partials) in the
// file-scope array below instead of a caller workspace.  The array is sized
// for the largest degree and grid, so every call of lsefit_fit fits in it.
// Every GPU that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------
namespace lsefit {

constexpr size_t kNoallocScratchBytes = 819456;  // kAlign + kMaxGrid * (3*8+1) * 8
static_assert(kNoallocScratchBytes >= kAlign + (size_t)kMaxGrid * (3 * LSEFIT_MAX_DEGREE + 1) * sizeof(double),
              "allocation-free scratch must hold the partials of the largest degree and grid");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch in the current context.  In host code
// the symbol names a host-side stand-in, not device memory, so the address is
// looked up (with the device current) and cached.  The cache is keyed by
// device and by the current driver context: a context that was torn down and
// created again (cudaDeviceReset, or another library resetting the primary
// context) holds the array at another address, so a new context makes the
// next call look the address up again.
typedef int (*ctx_get_current_t)(void** ctx);  // cuCtxGetCurrent(CUcontext*)

static ctx_get_current_t ctx_get_current() {
    static ctx_get_current_t fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<ctx_get_current_t>(p);
        (void)cudaGetLastError();
    });
    return fn;
}

static int noalloc_scratch(void** out) {
    static std::mutex mu;
    static void* addr[256] = {nullptr};
    static void* ctx_of[256] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        (void)cudaGetLastError();
        return LSEFIT_ERR_CUDA;
    }
    // the symbol lookup also makes the device's primary context current
    void* ctx = nullptr;
    ctx_get_current_t get = ctx_get_current();
    std::lock_guard<std::mutex> lock(mu);
    if (get != nullptr && (get(&ctx) != 0 || ctx == nullptr)) ctx = nullptr;
    if (addr[dev] == nullptr || ctx == nullptr || ctx != ctx_of[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return LSEFIT_ERR_CUDA;
        }
        if (get != nullptr && ctx == nullptr && (get(&ctx) != 0)) ctx = nullptr;
        addr[dev] = p;
        ctx_of[dev] = ctx;
    }
    *out = addr[dev];
    return LSEFIT_OK;
}

}  // namespace lsefit

extern "C" size_t lsefit_fit_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

extern "C" int lsefit_fit_noalloc(const void* x, const void* y, int64_t n, int dtype, int m, int m_lo,
                                  int accum, const double* interval, double* X, double* Xt, double* sums,
                                  double* map, int32_t* status, lsefit_stream_t stream) {
    if (m < 1 || m > LSEFIT_MAX_DEGREE) return LSEFIT_ERR_INVALID_ARG;
    if (lsefit_powersums_workspace_size(m) > kNoallocScratchBytes) return LSEFIT_ERR_SCRATCH_LIMIT;
    void* ws = nullptr;
    const int rc = noalloc_scratch(&ws);
    if (rc != LSEFIT_OK) return rc;
    // the ticket word must start at zero (each call also leaves it zeroed)
    if (cudaMemsetAsync(ws, 0, kAlign, (cudaStream_t)stream) != cudaSuccess) {
        (void)cudaGetLastError();  // the next call must not see this failure as its own
        return LSEFIT_ERR_CUDA;
    }
    return lsefit_fit(x, y, n, dtype, m, m_lo, accum, interval, X, Xt, sums, map, status, ws,
                      kNoallocScratchBytes, stream);
}
