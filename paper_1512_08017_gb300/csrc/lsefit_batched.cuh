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
// Persistent blocks (one per SM: the warp rings take most of its shared
// memory) take block tasks from an atomic queue until it is
// empty.  Then every warp takes warp tasks from a second atomic queue, in
// plan order (longest first, grouped by degree when the plan had degrees),
// drawing each index three tasks ahead so that its record, degree and map
// constants are loaded before they are needed.  A warp streams its
// series through a ring of shared-memory stages filled by cp.async copies
// that run ahead across task boundaries, so the bytes in flight do not
// depend on registers or on the length of the current series.
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

#ifndef LSEFIT_BATCHED_BLOCK
#define LSEFIT_BATCHED_BLOCK 512
#endif
constexpr int kBBlock = LSEFIT_BATCHED_BLOCK;  // threads of a persistent block (one per SM)
constexpr int kBWarps = kBBlock / 32;
constexpr int kDefaultWarpMaxLen = 65536;
constexpr int kDefaultChunkLen = 65536;

constexpr int kClasses = LSEFIT_MAX_DEGREE + 1;  // degree classes of the warp tasks
constexpr int kCounters = 3 + kClasses;          // queue counters in the workspace

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
    const int4* warp_tasks;   // {series, first point (low, high 32 bits), length}
    int n_warp_tasks;
    int64_t total_points;
    int sched;             // 1 one queue, 2 snake order, 3 degree classes
    int cls_begin[LSEFIT_MAX_DEGREE + 2];  // warp tasks of class c: [cls_begin[c], cls_begin[c+1])
    int cls_block[LSEFIT_MAX_DEGREE + 2];  // blocks starting on class c: [cls_block[c], cls_block[c+1])
    double* X;
    double* Xt;
    double* sums;
    double* map;
    int32_t* status;
    double eps;            // singularity threshold epsilon of the accumulation
    double* partials;      // [n_block_tasks][3*m_max+1]
    unsigned* tickets;     // [n_block_tasks], slot of a split series = its first task
    unsigned* counters;    // [0] block queue, [1] warp queue, [2] exited blocks, [3 + c] class c queue
    double2* mapc;         // [num_series]: FP32 paths {float2(c, s), unused}; FP64 {c, s}
    unsigned char* pend;   // [grid * kBWarps] queues of finished series
};

// ---------------------------------------------------------------------------
// preparation launch: clears the queue counters and split-series tickets, and
// computes the map constants of every series (one per thread).  Clearing here
// means the workspace needs no initialization and may be shared by plans of
// different layouts.
// ---------------------------------------------------------------------------
template <bool FP32MAP>
__global__ void batched_prep_kernel(__grid_constant__ const BParams p) {
    griddep_launch_dependents();  // the persistent kernel may start its set-up now
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < kCounters) p.counters[s] = 0u;
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
    // per warp, in the workspace: rows [32][kStride] words, then sid[32], meta[32]
    static constexpr size_t kWarpBytes = (size_t)32 * kStride * 8 + 32 * 4 * 2;
};

// A warp's queue of finished series.  The entry count n is warp-uniform
// register state, updated identically by every lane of the owning warp (no
// lane ever waits on another lane's store to learn it); it is published to
// shared memory only for the block's final consolidated solve.
template <int NMAX>
struct Pend {
    unsigned long long* row;  // [32][kStride] 8-byte words (global workspace)
    int* sid;                 // [32] series id (global workspace)
    int* meta;                // [32] degree (global workspace)
    int n;                    // entries queued
    __device__ __forceinline__ void bind(unsigned char* base) {
        row = reinterpret_cast<unsigned long long*>(base);
        sid = reinterpret_cast<int*>(base + 32 * PendLayout<NMAX>::kStride * 8);
        meta = sid + 32;
        n = 0;
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

// ---------------------------------------------------------------------------
// Warp stage rings (phase 2).  Stage boundaries lie on a fixed grid of
// kStageBytes in the concatenated arrays, so every stage is a slice of one
// aligned block and all but the first and last stage of a series are full.
// ---------------------------------------------------------------------------
#ifndef LSEFIT_RING_STAGES
#define LSEFIT_RING_STAGES 3
#endif
#ifndef LSEFIT_STAGE_BYTES
#define LSEFIT_STAGE_BYTES 2048
#endif
#ifndef LSEFIT_FOLD_STAGES
#define LSEFIT_FOLD_STAGES 2
#endif
constexpr int kRing = LSEFIT_RING_STAGES;        // stages per warp ring
constexpr int kStageBytes = LSEFIT_STAGE_BYTES;  // bytes of x (and of y) per stage
constexpr int kStageVecs = kStageBytes / 16;     // 16-byte vectors per stage (4 per lane)
constexpr int kFoldStages = LSEFIT_FOLD_STAGES;  // compensated batch = this many stages
static_assert(kRing >= 2 && kRing <= 3 && kStageVecs % 32 == 0, "ring geometry");
#ifndef LSEFIT_STAGE_UNROLL
#define LSEFIT_STAGE_UNROLL 1
#endif
// Vectors of a stage a lane handles per loop iteration.  Kept small: every
// degree has its own copy of the loop, and the warps of an SM that work on
// different degrees share its instruction caches.
constexpr int kStageUnroll = LSEFIT_STAGE_UNROLL;
constexpr int kBlockUnroll = 2;                  // vectors in flight per thread in block tasks

struct __align__(16) StageRec {
    long long r0;   // first point of the stage
    int n;          // points in the stage
    int s;          // series
    int flags;      // 1: first stage of the series, 2: last stage
    int deg;        // degree of the series
    double2 map;    // prepared map constants (raw 16 bytes, see batched_prep_kernel)
};

constexpr int kRingWarpBytes = 2 * kRing * kStageBytes + kRing * (int)sizeof(StageRec);

// Shared memory: [block-reduction scratch | warp rings] (phases 1 and 2 never
// overlap), blk, comb and the queue counts; the queues of finished series
// live in the workspace (written and read once per series).
constexpr size_t kRedBytes = (size_t)kBWarps * kBBlock * 8;
constexpr size_t kRingsBytes = (size_t)kBWarps * kRingWarpBytes;
constexpr size_t kScratchBytes = kRedBytes > kRingsBytes ? kRedBytes : kRingsBytes;

__host__ __device__ constexpr size_t batched_smem_bytes(int /*nmax*/) {
    return kScratchBytes + 32 * 8 /* blk */ + 32 * 8 /* comb */ + kBWarps * 4 /* queue counts */;
}

__host__ __device__ constexpr size_t pend_warp_bytes(int nmax) {
    return (size_t)32 * (3 * nmax + 2) * 8 + 32 * 4 * 2;
}

struct Ring {
    unsigned char* x;  // [kRing][kStageBytes]
    unsigned char* y;  // [kRing][kStageBytes]
    StageRec* rec;     // [kRing]
    __device__ __forceinline__ void bind(unsigned char* base) {
        x = base;
        y = base + kRing * kStageBytes;
        rec = reinterpret_cast<StageRec*>(base + 2 * kRing * kStageBytes);
    }
};

// Producer cursor of a warp.  Warp tasks are drawn from one queue in plan
// order (schedule 1), in a fixed snake order (schedule 2: round r gives warp
// w task r*W + w, or r*W + W-1-w on odd rounds, W warps in the grid numbered
// warp-major, w = warp * blocks + block, so that a round that is only partly
// filled still gives every SM the same share), or
// from one queue per degree class (schedule 3): a block starts on the class
// its index falls in when the blocks are shared out in proportion to the
// classes' cost, points x cost per point of the degree (cls_block, set at
// launch), and a warp whose class has run dry moves on to the next class with
// tasks left, so the warps of an SM keep running the code of one degree.  In schedules 1 and 3 the first
// kStaticRounds draws of a warp are fixed snake rounds over the warps of its
// first queue (numbered warp-major too) and only later draws take an atomic
// ticket (offset past the static rounds): a grid that starts with every warp hitting one counter
// spends microseconds in its queue.  Three tasks are in the pipeline ahead
// of the one being issued, one step per advance, so no advance waits on a
// load: tq (lane 0) holds the next index, a (lane 0) the task record loaded
// for the index before, b (all lanes) a record with its degree and map
// constants loaded.
struct Cursor {
    bool have;
    int s, deg;
    long long pos, end;
    double2 map;
    bool first;
    bool bv;
    int4 brec;
    int bdeg;
    double2 bmap;
    int at;     // lane 0: task index of slot a (>= n_warp_tasks: none)
    int4 arec;  // lane 0: record of slot a
    int tq;     // lane 0: next task index
    int round;  // lane 0: snake round of the next index (static rounds while < kStaticRounds)
    int cls;    // lane 0: queue drawn from (degree class; 0 in schedule 1)
};

constexpr int kStaticRounds = 3;
constexpr int kOwnSolveMin = 16;  // queue entries from which a warp solves its own queue after its stream

// Returns {task index (kNone: no work left), round, queue} for the draw made
// in state (round, cls).  Out of line, with the state passed by value, so the
// cursor itself stays in registers.
static __device__ __noinline__ int3 cursor_draw(int round, int cls, const BParams& p) {
    constexpr int kNone = 0x7fffffff;
    const int warp = threadIdx.x >> 5;
    if (p.sched == 2) {
        const long long nw = (long long)gridDim.x * kBWarps;
        // warp-major numbering: consecutive indices go to the same warp slot of
        // consecutive blocks, so a partly filled round is spread over every SM
        const long long wid = (long long)warp * gridDim.x + blockIdx.x;
        const long long t = (long long)round * nw + ((round & 1) ? (nw - 1 - wid) : wid);
        round++;
        return make_int3(t < p.n_warp_tasks ? (int)t : kNone, round, cls);
    }
    const bool classes = p.sched == 3;
    // every queue is visited at most once per draw; a queue stays behind once it runs dry
    for (int tries = 0; tries <= kClasses; ++tries) {
        const int c = cls;
        const int b = classes ? p.cls_begin[c] : 0;
        const int n = classes ? p.cls_begin[c + 1] - b : p.n_warp_tasks;
        const int blk0 = classes ? p.cls_block[c] : 0;
        const int nwc = (classes ? p.cls_block[c + 1] - blk0 : (int)gridDim.x) * kBWarps;
        const int nstatic = min(n, kStaticRounds * nwc);
        if (round < kStaticRounds) {  // the warp's first queue: fixed snake rounds
            const int nblk = nwc / kBWarps;
            const int r = warp * nblk + ((int)blockIdx.x - blk0);  // warp-major, as in schedule 2
            const int local = round * nwc + ((round & 1) ? (nwc - 1 - r) : r);
            round++;
            if (local < nstatic) return make_int3(b + local, round, cls);
            round = kStaticRounds;
        }
        if (n > nstatic) {
            const unsigned k = atomicAdd(&p.counters[classes ? 3 + c : 1], 1u);
            if (k < (unsigned)(n - nstatic)) return make_int3(b + nstatic + (int)k, round, cls);
        }
        if (!classes) return make_int3(kNone, round, cls);
        cls = c + 1 == kClasses ? 0 : c + 1;
        round = kStaticRounds;
    }
    return make_int3(kNone, round, cls);
}

// First queue of this block's warps: the degree class whose block range holds
// blockIdx.x (schedule 3), else the single queue.
__device__ __forceinline__ int first_class(const BParams& p) {
    if (p.sched != 3) return 0;
    for (int c = 0; c < kClasses; ++c)
        if ((int)blockIdx.x < p.cls_block[c + 1]) return c;
    return 0;
}

// One step of the pipeline: b becomes current, a moves to b (loading degree
// and map), the queued index moves to a (loading its record), and a new
// index is drawn.  Tasks of an invalid degree are marked and skipped.
__device__ __forceinline__ void cursor_step(Cursor& cu, const BParams& p) {
    const int lane = threadIdx.x & 31;
    cu.have = cu.bv;
    if (cu.have) {
        cu.s = cu.brec.x;
        cu.pos = ((long long)(unsigned)cu.brec.z << 32) | (unsigned)cu.brec.y;
        cu.end = cu.pos + cu.brec.w;
        cu.deg = cu.bdeg;
        cu.map = cu.bmap;
        cu.first = true;
    }
    const int at = __shfl_sync(0xffffffffu, cu.at, 0);
    cu.bv = at < p.n_warp_tasks;
    if (cu.bv) {
        cu.brec.x = __shfl_sync(0xffffffffu, cu.arec.x, 0);
        cu.brec.y = __shfl_sync(0xffffffffu, cu.arec.y, 0);
        cu.brec.z = __shfl_sync(0xffffffffu, cu.arec.z, 0);
        cu.brec.w = __shfl_sync(0xffffffffu, cu.arec.w, 0);
        cu.bdeg = p.degree[cu.brec.x];
        cu.bmap = p.mapc[cu.brec.x];
    }
    if (lane == 0) {
        cu.at = cu.tq;
        if (cu.tq < p.n_warp_tasks) {
            cu.arec = p.warp_tasks[cu.tq];
            const int3 d = cursor_draw(cu.round, cu.cls, p);
            cu.tq = d.x;
            cu.round = d.y;
            cu.cls = d.z;
        }
    }
}

// Status and NaN row of the cursor's current task, whose degree is outside
// 1..m_max: it is not fitted at all and gets no stages (lane 0 writes).
__device__ __forceinline__ void mark_invalid_task(const Cursor& cu, const BParams& p) {
    if ((threadIdx.x & 31) == 0) {
        const int64_t s = cu.s;
        const int nc = p.m_max + 1;
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        for (int i = 0; i < nc; ++i) {
            p.X[s * nc + i] = qnan;
            if (p.Xt) p.Xt[s * nc + i] = qnan;
        }
        if (p.sums)
            for (int k = 0; k < 3 * p.m_max + 2; ++k) p.sums[s * (3 * p.m_max + 2) + k] = qnan;
        p.status[s] = LSEFIT_ERR_INVALID_ARG;
    }
}

__device__ __forceinline__ bool cursor_valid_degree(const Cursor& cu, const BParams& p) {
    return cu.deg >= 1 && cu.deg <= p.m_max;
}

__device__ __forceinline__ void cursor_advance(Cursor& cu, const BParams& p) {
    for (;;) {
        cursor_step(cu, p);
        if (!cu.have || cursor_valid_degree(cu, p)) return;
        mark_invalid_task(cu, p);
    }
}

// Start of phase 2: the first draw, then one pipeline step per prefetch slot
// (index -> a -> b -> current).
__device__ __forceinline__ void cursor_init(Cursor& cu, const BParams& p) {
    cu.have = false;
    cu.bv = false;
    cu.at = 0x7fffffff;
    cu.arec = make_int4(0, 0, 0, 0);
    cu.tq = 0x7fffffff;
    cu.round = 0;
    cu.cls = 0;
    // map constants and queue counters come from the preparation launch (a
    // first draw can already reach an atomic queue when its static round is
    // empty)
    griddep_wait();
    if ((threadIdx.x & 31) == 0) {
        const int3 d = cursor_draw(0, first_class(p), p);
        cu.tq = d.x;
        cu.round = d.y;
        cu.cls = d.z;
    }
    cursor_step(cu, p);     // index -> a
    cursor_step(cu, p);     // a -> b
    cursor_advance(cu, p);  // b -> current
}

template <int ES>
__device__ __forceinline__ void copy_elem(unsigned char* dst, const unsigned char* src) {
    if (ES == 2) *reinterpret_cast<unsigned short*>(dst) = *reinterpret_cast<const unsigned short*>(src);
    else if (ES == 4) *reinterpret_cast<unsigned*>(dst) = *reinterpret_cast<const unsigned*>(src);
    else *reinterpret_cast<unsigned long long*>(dst) = *reinterpret_cast<const unsigned long long*>(src);
}

// Issue the next stage of the cursor's series into ring slot `slot` (all
// lanes; one commit group per call).  Returns false when the warp has no
// work left.
template <int DT>
__device__ __forceinline__ bool issue_stage(const BParams& p, Ring& R, int slot, Cursor& cu) {
    if (!cu.have) return false;
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec, P = kStageBytes / ES;
    const int lane = threadIdx.x & 31;
    const long long r0 = cu.pos;
    const long long r1 = min(cu.end, (r0 / P + 1) * P);
    const long long g0 = r0 & ~(long long)(PV - 1);
    const long long gend = (r1 + PV - 1) & ~(long long)(PV - 1);
    const int nv = (int)((gend - g0) / PV);
    unsigned char* xb = R.x + slot * kStageBytes;
    unsigned char* yb = R.y + slot * kStageBytes;
    const unsigned char* xg = static_cast<const unsigned char*>(p.x) + g0 * ES;
    const unsigned char* yg = static_cast<const unsigned char*>(p.y) + g0 * ES;
    if (gend <= p.total_points) {
        for (int v = lane; v < nv; v += 32) {
            cp_async16(xb + 16 * v, xg + 16 * v);
            cp_async16(yb + 16 * v, yg + 16 * v);
        }
    } else for (int v = lane; v < nv; v += 32) {
        if (g0 + (long long)(v + 1) * PV <= p.total_points) {
            cp_async16(xb + 16 * v, xg + 16 * v);
            cp_async16(yb + 16 * v, yg + 16 * v);
        } else {
            // the vector that crosses the end of the arrays: element by element
            for (int u = 0; u < PV; ++u) {
                if (g0 + (long long)v * PV + u < p.total_points) {
                    copy_elem<ES>(xb + 16 * v + u * ES, xg + 16 * v + u * ES);
                    copy_elem<ES>(yb + 16 * v + u * ES, yg + 16 * v + u * ES);
                }
            }
        }
    }
    cp_async_commit();
    if (lane == 0) {
        StageRec& rc = R.rec[slot];
        rc.r0 = r0;
        rc.n = (int)(r1 - r0);
        rc.s = cu.s;
        rc.flags = (cu.first ? 1 : 0) | (r1 == cu.end ? 2 : 0);
        rc.deg = cu.deg;
        rc.map = cu.map;
    }
    cu.first = false;
    cu.pos = r1;
    if (r1 == cu.end) cursor_advance(cu, p);
    return true;
}

// Wait until the oldest of `pending` stages has landed, then make every
// lane's copies visible to the warp.
__device__ __forceinline__ void ring_wait(int pending) {
    static_assert(kRing <= 3, "ring_wait covers up to three pending stages");
    switch (pending) {
        case 1: cp_async_wait<0>(); break;
        case 2: cp_async_wait<1>(); break;
        default: cp_async_wait<2>(); break;
    }
    __syncwarp();
}

// Solve one queued series (entry idx of warp ws's queue in this block), if
// `active`.  Called by all 32 lanes of a warp together (the degree and map
// votes below span the full warp).  Converts the entry's sums to FP64 in place.
template <int NMAX, int ACC, bool CHEB = false>
__device__ __noinline__ void pend_solve_entry(const BParams& p, unsigned char* pend_block, int ws, int idx,
                                              bool active) {
    constexpr int W = PendLayout<NMAX>::kStride;
    int m = 0;
    int64_t s = 0;
    double c = 0.0, sc = 1.0;
    bool ok = false;
    double* sm = nullptr;
    if (active) {
        unsigned char* base = pend_block + (size_t)ws * PendLayout<NMAX>::kWarpBytes;
        unsigned long long* row = reinterpret_cast<unsigned long long*>(base) + (size_t)idx * W;
        const int* sid = reinterpret_cast<const int*>(base + 32 * W * 8);
        m = sid[32 + idx];
        s = sid[idx];
        const int ns = 3 * m + 2;
        if (ACC == LSEFIT_ACCUM_F64) {
            ok = load_map_f64(p, s, c, sc);
        } else {
            float cf, sf;
            ok = load_map_f32(p, s, cf, sf);
            c = f32_to_f64_int(cf);
            sc = f32_to_f64_int(sf);
        }
        // the sums output (monomial basis) is stored as the sums are converted,
        // so that its stores drain during the elimination; the Chebyshev moments
        // are only final after the solve's fix-up and are stored there
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        const int stride = 3 * p.m_max + 2;
        double* so = (!CHEB && p.sums) ? p.sums + s * stride : nullptr;
        sm = reinterpret_cast<double*>(row);
        sm[0] = (double)(long long)row[0];
        if (so) so[0] = ok ? sm[0] : qnan;
        if (ACC != LSEFIT_ACCUM_F64) {
            for (int k = 1; k < ns; ++k) {
                const dflt v = bits_df(row[k]);
                const double d = f32_to_f64_int(v.hi) + f32_to_f64_int(v.lo);
                sm[k] = d;
                if (so) so[k] = ok ? d : qnan;
            }
        } else if (so) {
            for (int k = 1; k < ns; ++k) so[k] = ok ? sm[k] : qnan;
        }
        if (so)
            for (int k = ns; k < stride; ++k) so[k] = 0.0;
    }
    // the solve is sized for the largest degree among the lanes solving together
    // (FP64 instructions cost the same for 1 or 32 lanes; padding does not), and
    // skips the un-map when every lane's map is the identity (c = 0, s = 1)
    const int mw = (int)__reduce_max_sync(0xffffffffu, active ? (unsigned)m : 0u);
    const bool id = __all_sync(0xffffffffu, !active || (__double_as_longlong(c) == 0ll &&
                                                        __double_as_longlong(sc) == 0x3ff0000000000000ll));
    if (!active) return;
    const int nc = p.m_max + 1;
    double* xt = p.Xt ? p.Xt + s * nc : nullptr;
    double* x = p.X + s * nc;
    const double* T = sm + 2 * m + 1;
    int st;
    if (CHEB && active) cheb_moments_from_products(m, sm);  // degrees m+1..2m were kept as product sums
    if (CHEB) {
        // Chebyshev basis: G from the moments (sm[0] = n), Xt holds the Chebyshev coefficients
        switch (mw) {
            case 1: st = solve_general_rt<1, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
            case 2: st = solve_general_rt<2, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
            case 3: st = solve_general_rt<3, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
            case 4: st = solve_general_rt<4, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
            default:
                if constexpr (NMAX > 5) {
                    switch (mw) {
                        case 5: st = solve_general_rt<5, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
                        case 6: st = solve_general_rt<6, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
                        case 7: st = solve_general_rt<7, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
                        default: st = solve_general_rt<8, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc); break;
                    }
                } else {
                    st = solve_general_rt<5, true>(m, sm, T, sm[0], c, sc, ok, p.eps, xt, x, nc);
                }
                break;
        }
    } else
    switch (mw) {
        case 1: st = solve_hankel_rt<1>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
        case 2: st = solve_hankel_rt<2>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
        case 3: st = solve_hankel_rt<3>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
        case 4: st = solve_hankel_rt<4>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
        default:
            if constexpr (NMAX > 5) {
                switch (mw) {
                    case 5: st = solve_hankel_rt<5>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
                    case 6: st = solve_hankel_rt<6>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
                    case 7: st = solve_hankel_rt<7>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
                    default: st = solve_hankel_rt<8>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id); break;
                }
            } else {
                st = solve_hankel_rt<5>(m, sm, T, c, sc, ok, p.eps, xt, x, nc, id);
            }
            break;
    }
    p.status[s] = st;
    if (CHEB && p.sums) {
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        const int stride = 3 * p.m_max + 2;
        const int ns = 3 * m + 2;
        double* out = p.sums + s * stride;
        for (int k = 0; k < stride; ++k) out[k] = k < ns ? (ok ? sm[k] : qnan) : 0.0;
    }
}

// The warp solves its full queue (32 series), one per lane, and empties it.
template <int NMAX, int ACC, bool CHEB = false>
__device__ __forceinline__ void pend_solve(const BParams& p, Pend<NMAX>& q) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    unsigned char* base = reinterpret_cast<unsigned char*>(q.row);
    // the queue of warp w of this block is at pend_block + w * kWarpBytes; solve
    // entries relative to this warp's own queue
    pend_solve_entry<NMAX, ACC, CHEB>(p, base, 0, lane, lane < q.n);
    __syncwarp();
    q.n = 0;
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
template <int NMAX, int DT, int ACC, int M, bool CHEB = false>
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
        AccF64<M, CHEB> A;
        A.init();
        if (ok) accumulate_range_f64<M, DT, kBlockUnroll, true, CHEB>(A, p.x, p.y, b, e, tid, kBBlock, c, sc);
        block_reduce_d<kBBlock, N>([&](int a) { return A.acc[a]; }, reinterpret_cast<double*>(red), blk);
        // blk[a] (doubles) == words[a]
    } else {
        float c, sc;
        const bool ok = load_map_f32(p, s, c, sc);
        AccF32<M, ACC == LSEFIT_ACCUM_COMP, true, CHEB> A;
        A.init();
        if (ok) accumulate_range<M, DT, ACC == LSEFIT_ACCUM_COMP, true, kBlockUnroll, true, CHEB>(
            A, p.x, p.y, b, e, tid, kBBlock, c, sc);
        block_reduce_df2<kBBlock, N>([&](int a) { return A.result(a); }, red, reinterpret_cast<dflt*>(blk));
    }
    // words[0..N-1] now hold this chunk's totals (visible to all threads)
    const int slot_row = PendLayout<NMAX>::kStride;
    if (nch == 1) {
        if (tid == 0) {
            const int slot = q0.n;
            unsigned long long* row = q0.row + slot * slot_row;
            row[0] = (unsigned long long)len;
            for (int a = 0; a < N; ++a) row[a + 1] = words[a];
            q0.sid[slot] = (int)s;
            q0.meta[slot] = M;
        }
        if (tid < 32) q0.n += 1;
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
                const int slot = q0.n;
                unsigned long long* row = q0.row + slot * slot_row;
                row[0] = (unsigned long long)len;
                for (int a = 0; a < N; ++a) row[a + 1] = reinterpret_cast<unsigned long long*>(comb)[a];
                q0.sid[slot] = (int)s;
                q0.meta[slot] = M;
                p.tickets[first] = 0u;
            }
            if (tid < 32) q0.n += 1;
        }
    }
    if (tid < 32) {
        __syncwarp();
        if (q0.n == 32) pend_solve<NMAX, ACC, CHEB>(p, q0);
    }
}

// ---------------------------------------------------------------------------
// Accumulation of one stage from shared memory.  Buffer element j holds point
// g0 + j (g0: r0 rounded down to a 16-byte vector); points outside
// [r0, r0 + n) are masked out.
// ---------------------------------------------------------------------------
// Zero the pair (t, y) where its element index e (first of the pair) is
// outside [lo, hi): a zero abscissa and ordinate add nothing to the sums of
// degree >= 1 (S_0 is the count, kept apart).
__device__ __forceinline__ void mask_pair(u64& t, u64& y, u64& seed, int e, int lo, int hi) {
    float t0, t1, y0, y1;
    up2(t, t0, t1);
    up2(y, y0, y1);
    const bool ok0 = e >= lo && e < hi, ok1 = e + 1 >= lo && e + 1 < hi;
    t = pk2(ok0 ? t0 : 0.0f, ok1 ? t1 : 0.0f);
    y = pk2(ok0 ? y0 : 0.0f, ok1 ? y1 : 0.0f);
    seed = pk2(ok0 ? 1.0f : 0.0f, ok1 ? 1.0f : 0.0f);
}

// Accumulate the points [lo, hi) of one landed stage (element indices
// relative to the stage's first vector).  Full vectors and the partial first
// and last vectors of a series take the same packed code; a partial vector
// only masks its pairs.
template <int M, int DT, bool COMP, bool SHL, bool CHEB = false>
__device__ __forceinline__ void stage_accumulate_f32(AccF32<M, COMP, SHL, CHEB>& A, const unsigned char* xb,
                                                     const unsigned char* yb, long long r0, int n, float cf,
                                                     float sf) {
    constexpr int PV = Elem<DT>::kPerVec, P = kStageBytes / Elem<DT>::kSize;
    const int lane = threadIdx.x & 31;
    const int lo = (int)(r0 & (PV - 1));
    const int hi = lo + n;
    const int nv = (hi + PV - 1) / PV;
    const u64 c2 = pk2(cf, cf), s2 = pk2(sf, sf);
    const bool full = (lo == 0 && n == P);
#pragma unroll kStageUnroll
    for (int q = 0; q < kStageVecs / 32; ++q) {
        const int v = lane + 32 * q;
        if (v >= nv) break;
        const uint4 xv = *reinterpret_cast<const uint4*>(xb + 16 * v);
        const uint4 yv = *reinterpret_cast<const uint4*>(yb + 16 * v);
        const bool part = !full && (v * PV < lo || (v + 1) * PV > hi);
        const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
        const uint32_t yw[4] = {yv.x, yv.y, yv.z, yv.w};
        constexpr int NPAIR = PV / 2;
#pragma unroll
        for (int k = 0; k < NPAIR; ++k) {
            u64 tp, yp;
            if (DT == LSEFIT_F32) {
                tp = pk2(__uint_as_float(xw[2 * k]), __uint_as_float(xw[2 * k + 1]));
                yp = pk2(__uint_as_float(yw[2 * k]), __uint_as_float(yw[2 * k + 1]));
            } else {
                tp = pk2(bf16_lo(xw[k]), bf16_hi(xw[k]));
                yp = pk2(bf16_lo(yw[k]), bf16_hi(yw[k]));
            }
            tp = mul2(sub2(tp, c2), s2);
            u64 seed = CHEB ? pk2(1.0f, 1.0f) : 0ull;
            if (part) mask_pair(tp, yp, seed, v * PV + 2 * k, lo, hi);
            A.template add_pair<false>(tp, yp, seed);
        }
    }
}

template <int M, int DT, bool CHEB = false>
__device__ __forceinline__ void stage_accumulate_f64(AccF64<M, CHEB>& A, const unsigned char* xb,
                                                     const unsigned char* yb, long long r0, int n, double c,
                                                     double sc) {
    constexpr int PV = Elem<DT>::kPerVec;
    const int lane = threadIdx.x & 31;
    const int lo = (int)(r0 & (PV - 1));
    const int hi = lo + n;
    const int nv = (hi + PV - 1) / PV;
#pragma unroll
    for (int q = 0; q < kStageVecs / 32; ++q) {
        const int v = lane + 32 * q;
        if (v >= nv) continue;
        double xs[PV], ys[PV];
        unpack_f64<DT, PV>(*reinterpret_cast<const uint4*>(xb + 16 * v), xs);
        unpack_f64<DT, PV>(*reinterpret_cast<const uint4*>(yb + 16 * v), ys);
#pragma unroll
        for (int k = 0; k < PV; ++k) {
            const int e = v * PV + k;
            if (e >= lo && e < hi) A.add_point(sc * (xs[k] - c), ys[k]);
        }
    }
}

// One series streamed through the ring.  On entry the stage at `slot` is its
// first stage and has landed; on return `slot` is the stage after its last.
template <int NMAX, int DT, int ACC, int M, bool CHEB = false>
__device__ void ring_task(const BParams& p, Ring& R, int& slot, int& pending, Cursor& cu, Pend<NMAX>& q) {
    constexpr int N = 3 * M + 1;
    constexpr int NP = N <= 16 ? 16 : 32;
    const int lane = threadIdx.x & 31;
    const int s = R.rec[slot].s;
    const double2 mraw = R.rec[slot].map;
    long long count = 0;
    if constexpr (ACC == LSEFIT_ACCUM_F64) {
        const bool ok = !isnan(mraw.x);
        const double c = ok ? mraw.x : 0.0, sc = ok ? mraw.y : 1.0;
        AccF64<M, CHEB> A;
        A.init();
        for (;;) {
            const long long r0 = R.rec[slot].r0;
            const int n = R.rec[slot].n, flags = R.rec[slot].flags;
            if (ok) stage_accumulate_f64<M, DT, CHEB>(A, R.x + slot * kStageBytes, R.y + slot * kStageBytes, r0, n, c, sc);
            count += n;
            __syncwarp();
            --pending;
            if (issue_stage<DT>(p, R, slot, cu)) ++pending;
            slot = slot + 1 == kRing ? 0 : slot + 1;
            if (flags & 2) break;
            ring_wait(pending);
        }
        double v[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) v[a] = a < N ? A.acc[a] : 0.0;
        const double tot = warp_reduce_scatter_d<NP>(v);
        const int qs = q.n;
        unsigned long long* row = q.row + qs * PendLayout<NMAX>::kStride;
        if (lane < N) row[lane + 1] = (unsigned long long)__double_as_longlong(tot);
    } else {
        const float2 mf = *reinterpret_cast<const float2*>(&mraw);
        const bool ok = !isnan(mf.x);
        const float c = ok ? mf.x : 0.0f, sc = ok ? mf.y : 1.0f;
        AccF32<M, ACC == LSEFIT_ACCUM_COMP, true, CHEB> A;
        A.init();
        int since_fold = 0;
        for (;;) {
            const long long r0 = R.rec[slot].r0;
            const int n = R.rec[slot].n, flags = R.rec[slot].flags;
            if (ok)
                stage_accumulate_f32<M, DT, ACC == LSEFIT_ACCUM_COMP, true, CHEB>(A, R.x + slot * kStageBytes,
                                                                            R.y + slot * kStageBytes, r0, n, c, sc);
            if (++since_fold == kFoldStages) {
                A.fold_reset();
                since_fold = 0;
            }
            count += n;
            __syncwarp();
            --pending;
            if (issue_stage<DT>(p, R, slot, cu)) ++pending;
            slot = slot + 1 == kRing ? 0 : slot + 1;
            if (flags & 2) break;
            ring_wait(pending);
        }
        if (since_fold) A.fold_reset();
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
        const int qs = q.n;
        unsigned long long* row = q.row + qs * PendLayout<NMAX>::kStride;
        if (lane < N) row[lane + 1] = df_bits(tot);
    }
    if (lane == 0) {
        const int qs = q.n;
        q.row[qs * PendLayout<NMAX>::kStride] = (unsigned long long)count;
        q.sid[qs] = s;
        q.meta[qs] = M;
    }
    q.n += 1;
    __syncwarp();
    if (q.n == 32) pend_solve<NMAX, ACC, CHEB>(p, q);
}

template <int NMAX, int DT, int ACC, bool CHEB = false>
__device__ __forceinline__ void dispatch_ring(const BParams& p, int m, Ring& R, int& slot, int& pending,
                                              Cursor& cu, Pend<NMAX>& q) {
    switch (m) {
        case 1: ring_task<NMAX, DT, ACC, 1, CHEB>(p, R, slot, pending, cu, q); break;
        case 2: ring_task<NMAX, DT, ACC, 2, CHEB>(p, R, slot, pending, cu, q); break;
        case 3: ring_task<NMAX, DT, ACC, 3, CHEB>(p, R, slot, pending, cu, q); break;
        case 4: ring_task<NMAX, DT, ACC, 4, CHEB>(p, R, slot, pending, cu, q); break;
        case 5: ring_task<NMAX, DT, ACC, 5, CHEB>(p, R, slot, pending, cu, q); break;
        default:
            if constexpr (NMAX > 5) {
                switch (m) {
                    case 6: ring_task<NMAX, DT, ACC, 6, CHEB>(p, R, slot, pending, cu, q); break;
                    case 7: ring_task<NMAX, DT, ACC, 7, CHEB>(p, R, slot, pending, cu, q); break;
                    default: ring_task<NMAX, DT, ACC, 8, CHEB>(p, R, slot, pending, cu, q); break;
                }
            }
            break;
    }
}

template <int NMAX, int DT, int ACC, bool CHEB = false>
__device__ __forceinline__ void dispatch_block(const BParams& p, int t, int4 task, int m, dflt* red,
                                               double* blk, double* comb, Pend<NMAX>& q0, int* s_last) {
    switch (m) {
        case 1: block_task<NMAX, DT, ACC, 1, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
        case 2: block_task<NMAX, DT, ACC, 2, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
        case 3: block_task<NMAX, DT, ACC, 3, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
        case 4: block_task<NMAX, DT, ACC, 4, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
        case 5: block_task<NMAX, DT, ACC, 5, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
        default:
            if constexpr (NMAX > 5) {
                switch (m) {
                    case 6: block_task<NMAX, DT, ACC, 6, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
                    case 7: block_task<NMAX, DT, ACC, 7, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
                    default: block_task<NMAX, DT, ACC, 8, CHEB>(p, t, task, red, blk, comb, q0, s_last); break;
                }
            }
            break;
    }
}

template <int NMAX, int DT, int ACC, bool CHEB = false>
__global__ void __launch_bounds__(kBBlock, 1) batched_kernel(__grid_constant__ const BParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_task;
    __shared__ int s_last;
    dflt* red = reinterpret_cast<dflt*>(smem);
    double* blk = reinterpret_cast<double*>(smem + kScratchBytes);
    double* comb = blk + 32;
    int* counts = reinterpret_cast<int*>(comb + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* pend_block = p.pend + (size_t)blockIdx.x * kBWarps * PendLayout<NMAX>::kWarpBytes;
    // each warp's queue; block tasks queue their series in warp 0's (whose
    // threads alone touch it there, so its count stays in warp 0's registers)
    Pend<NMAX> q;
    q.bind(pend_block + warp * PendLayout<NMAX>::kWarpBytes);

    // phase 1: block tasks (their queue counter is cleared by the preparation launch)
    if (p.n_block_tasks > 0) griddep_wait();
    for (; p.n_block_tasks > 0;) {
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
        dispatch_block<NMAX, DT, ACC, CHEB>(p, t, task, m, red, blk, comb, q, &s_last);
    }
    // phase 2: warp tasks through the warp's stage ring
    {
        Ring R;
        R.bind(smem + warp * kRingWarpBytes);
        Cursor cu;
        cursor_init(cu, p);
        int pending = 0;
#pragma unroll
        for (int k = 0; k < kRing; ++k)
            if (issue_stage<DT>(p, R, k, cu)) ++pending;
        int slot = 0;
        while (pending > 0) {
            ring_wait(pending);
            dispatch_ring<NMAX, DT, ACC, CHEB>(p, R.rec[slot].deg, R, slot, pending, cu, q);
        }
    }
    // A warp that ends its stream with a well-filled queue solves it at once,
    // while the block's other warps are still streaming; the rest of the
    // block's queued series are solved together after the stream, 32 per warp
    // (a warp-solve costs the same FP64 instructions for 1 lane as for 32).
    if (q.n >= kOwnSolveMin) pend_solve<NMAX, ACC, CHEB>(p, q);
    // leftover queued series of all warps, solved 32 per warp across the block
    if (lane == 0) counts[warp] = q.n;
    __syncthreads();
    {
        int total = 0;
        for (int w = 0; w < kBWarps; ++w) total += counts[w];
        for (int base = warp * 32; base < total; base += kBWarps * 32) {
            const int g = base + lane;
            int ws = 0, idx = g;
            while (ws < kBWarps && idx >= counts[ws]) {
                idx -= counts[ws];
                ++ws;
            }
            __syncwarp();  // the entry solve votes across the full warp
            pend_solve_entry<NMAX, ACC, CHEB>(p, pend_block, ws, idx, g < total);
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&p.counters[2], 1u) == gridDim.x - 1) {
            for (int c = 0; c < kCounters; ++c) p.counters[c] = 0u;
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

// The Chebyshev-basis kernels (compensated FP32 and FP64 accumulation).
#define LSEFIT_BATCHED_INSTANTIATE_CHEB(NAME, DT, ACC)                                         \
    batched_kernel_t NAME(int nmax) {                                                         \
        return nmax <= 5 ? batched_kernel<5, DT, ACC, true> : batched_kernel<8, DT, ACC, true>; \
    }

batched_kernel_t batched_f32_naive(int nmax);
batched_kernel_t batched_f32_comp(int nmax);
batched_kernel_t batched_f32_f64(int nmax);
batched_kernel_t batched_bf16_naive(int nmax);
batched_kernel_t batched_bf16_comp(int nmax);
batched_kernel_t batched_bf16_f64(int nmax);
batched_kernel_t batched_f64_f64(int nmax);
batched_kernel_t batched_f32_comp_cheb(int nmax);
batched_kernel_t batched_bf16_comp_cheb(int nmax);
batched_kernel_t batched_f32_f64_cheb(int nmax);
batched_kernel_t batched_f64_f64_cheb(int nmax);

}  // namespace lsefit
