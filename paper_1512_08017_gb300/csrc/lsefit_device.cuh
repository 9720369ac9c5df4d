// lsefit_device.cuh -- device building blocks of the least-squares polynomial fit.
//
// The fit (Dasgupta, arXiv 1512.08017, Section II) needs, for every point,
// the powers t^k (k <= 2m) added into S_k and t^k y added into T_k, then
// the Hankel system A[j][k] = S_{j+k}, B[j] = T_j solved by Gaussian
// elimination.  This header holds:
//   * packed FP32 pair arithmetic (Blackwell add/sub/mul/fma .f32x2): two
//     points per instruction in the per-point loop;
//   * TwoSum / double-float helpers for compensated accumulation;
//   * point loaders for F32 / BF16 / F64 storage;
//   * the per-thread accumulator (naive FP32, compensated, FP64);
//   * the block reduction of accumulators (double-float, fixed order);
//   * the FP64 Hankel solve with partial pivoting and the un-map.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lsefit.h"

namespace lsefit {

typedef unsigned long long u64;

// ---------------------------------------------------------------------------
// Packed FP32 pairs.  Each lane of a pair is an independent IEEE RN operation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 pk2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(u64 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth's TwoSum, Dekker's Fast2Sum) and a
// double-float value hi + lo.  Intrinsics keep every step a single rounding.
// ---------------------------------------------------------------------------
struct dflt {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    dflt r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ dflt df_shfl_xor(dflt v, int mask) {
    dflt r;
    r.hi = __shfl_xor_sync(0xffffffffu, v.hi, mask);
    r.lo = __shfl_xor_sync(0xffffffffu, v.lo, mask);
    return r;
}

__device__ __forceinline__ double df_to_double(dflt v) { return (double)v.hi + (double)v.lo; }

// Exact FP32 -> FP64 conversion with integer operations (no FP64 pipe):
// rebias the exponent and widen the significand; zero, subnormal, Inf and
// NaN are handled by their encodings.
__device__ __forceinline__ double f32_to_f64_int(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned ex = (u >> 23) & 0xffu;
    unsigned long long man = u & 0x7fffffu;
    unsigned long long bits;
    if (ex == 0xffu) {
        bits = sign | (0x7ffull << 52) | (man << 29);  // Inf / NaN
    } else if (ex != 0u) {
        bits = sign | ((unsigned long long)(ex + 896u) << 52) | (man << 29);  // 896 = 1023 - 127
    } else if (man == 0ull) {
        bits = sign;  // signed zero
    } else {
        // subnormal FP32: normalise the significand (FP64 has the range)
        const int lz = __clzll(man) - 40;  // leading zeros within the 23-bit field
        man = (man << (lz + 1)) & 0x7fffffull;
        bits = sign | ((unsigned long long)(896u - lz) << 52) | (man << 29);
    }
    return __longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------------------
// BF16 helpers (bit operations; a bfloat16 is the top half of an FP32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

template <int DT>
struct Elem;
template <>
struct Elem<LSEFIT_F32> {
    typedef float T;
    static constexpr int kSize = 4;
    static constexpr int kPerVec = 4;  // points per 16-byte vector
    __device__ static __forceinline__ float ld(const void* p, int64_t i) {
        return __ldg(reinterpret_cast<const float*>(p) + i);
    }
    __device__ static __forceinline__ double ld64(const void* p, int64_t i) { return (double)ld(p, i); }
};
template <>
struct Elem<LSEFIT_BF16> {
    typedef uint16_t T;
    static constexpr int kSize = 2;
    static constexpr int kPerVec = 8;
    __device__ static __forceinline__ float ld(const void* p, int64_t i) {
        uint16_t b = __ldg(reinterpret_cast<const unsigned short*>(p) + i);
        return __uint_as_float(((uint32_t)b) << 16);
    }
    __device__ static __forceinline__ double ld64(const void* p, int64_t i) { return (double)ld(p, i); }
};
template <>
struct Elem<LSEFIT_F64> {
    typedef double T;
    static constexpr int kSize = 8;
    static constexpr int kPerVec = 2;
    __device__ static __forceinline__ double ld64(const void* p, int64_t i) {
        return __ldg(reinterpret_cast<const double*>(p) + i);
    }
};

// L2 policy of data read once: its lines are the first to be replaced.  A
// pass over more bytes than L2 holds would otherwise push out what the next
// launch needs at once (its code, plan and per-series records), and a launch
// of a few tens of microseconds then starts by waiting on DRAM for those.
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 16-byte vector load that is not kept in L1 and leaves L2 first (streamed once).
__device__ __forceinline__ uint4 ld_stream16(const void* p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(l2_evict_first_policy()));
    return r;
}

// L2 prefetch of [p, p + bytes): a hint with nothing to wait for, holding no
// registers (p 16-byte aligned, bytes a multiple of 16, the range inside one
// allocation).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch of the line that holds p (one thread's share of a coalesced prefetch).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ---------------------------------------------------------------------------
// Asynchronous global->shared copies (cp.async): in flight without holding
// registers; cp.async.wait_group is a hardware wait on this thread's groups.
// ---------------------------------------------------------------------------
// (the streamed inputs: L2 evict-first, as ld_stream16)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem_src),
                 "l"(l2_evict_first_policy())
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while the kernel before it on the stream is still
// running: griddep_wait() returns once that kernel has completed and its
// writes are visible (at once when the launch carries no such dependency),
// and griddep_launch_dependents() lets the kernel after this one start early.
// Both are hardware-managed: no thread spins on memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::); }

// ---------------------------------------------------------------------------
// Map constants.  c = (lo + hi) / 2, s = 2 / (hi - lo) in FP64, rounded once
// to FP32 when the points are mapped in FP32.  Identity without an interval.
// Returns false for an interval that is not finite or has hi <= lo.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool map_constants(const double* interval, bool fp32, double& c, double& s) {
    if (interval == nullptr) {
        c = 0.0;
        s = 1.0;
        return true;
    }
    const double lo = interval[0], hi = interval[1];
    if (!(isfinite(lo) && isfinite(hi)) || !(hi > lo)) {
        c = 0.0;
        s = 1.0;
        return false;
    }
    double cc = (lo + hi) * 0.5;
    double ss = 2.0 / (hi - lo);
    if (fp32) {
        cc = (double)__double2float_rn(cc);
        ss = (double)__double2float_rn(ss);
    }
    if (!isfinite(cc) || !isfinite(ss) || ss == 0.0) {
        c = 0.0;
        s = 1.0;
        return false;
    }
    c = cc;
    s = ss;
    return true;
}

// ---------------------------------------------------------------------------
// Per-thread accumulators for degree M.  Accumulator a: a < 2M holds S_{a+1},
// a >= 2M holds T_{a-2M}.  (S_0 is the exact point count, never summed.)
// ---------------------------------------------------------------------------
template <int M>
struct Nacc {
    static constexpr int value = 3 * M + 1;
};

// FP32 pair accumulator: each u64 carries two independent lane sums.
// COMP adds a TwoSum pair (hi, lo) per accumulator, fed once per batch:
//  * SHL = false: (hi, lo) are packed pairs too, one per lane (6 registers per
//    accumulator; the fold is 7 packed instructions);
//  * SHL = true: (hi, lo) are scalars; the two lanes of the batch sum are
//    added first (one rounding of the batch's own size), then added to hi
//    exactly (4 registers per accumulator; 8 scalar instructions).
// CHEB: the basis values are the Chebyshev polynomials T_k(t) (recurrence
// T_{k+1} = 2t T_k - T_{k-1}) instead of the powers t^k; the slots keep the
// same layout (moments of degree 1..2M, then the right-hand sides).  The
// values are carried as sigma_k T_k, sigma_k = -1 for k = 2, 3 (mod 4) and +1
// otherwise, which makes each step one fma with +-2t and no negation
// (sigma_{k+1} sigma_{k-1} = -1); rounding to nearest is symmetric under
// negation, and result() restores the sign.
template <int M, bool COMP, bool SHL = false, bool CHEB = false>
struct AccF32 {
    static constexpr int N = 3 * M + 1;
    u64 acc[N];
    u64 phi[(COMP && !SHL) ? N : 1], plo[(COMP && !SHL) ? N : 1];
    float shi[(COMP && SHL) ? N : 1], slo[(COMP && SHL) ? N : 1];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int a = 0; a < N; ++a) acc[a] = 0ull;
        if (COMP && !SHL) {
#pragma unroll
            for (int a = 0; a < N; ++a) {
                phi[a] = 0ull;
                plo[a] = 0ull;
            }
        }
        if (COMP && SHL) {
#pragma unroll
            for (int a = 0; a < N; ++a) {
                shi[a] = 0.0f;
                slo[a] = 0.0f;
            }
        }
    }

    // Add the two points (t.x, y.x), (t.y, y.y).  FIRST assigns instead of
    // adding (the first pair of a compensated batch).  seed: 1 per valid lane,
    // 0 for an empty lane (read only by the Chebyshev recurrence, whose
    // T_0 = 1 would otherwise make an empty lane with t = 0 count in T_2).
    template <bool FIRST>
    __device__ __forceinline__ void add_pair(u64 t, u64 y, u64 seed = 0ull) {
        if (!CHEB) {
            add_pair_powers<FIRST>(t, y);
            return;
        }
        // Chebyshev: v_k = sigma_k T_k by the recurrence up to k = M feeds the
        // moments of degree 1..M and the right-hand sides; the slot of degree
        // k = M+1..2M takes the product v_a v_b (a = k/2, b = k - a), whose sum
        // is sigma_a sigma_b (C_k + C_{b-a}) / 2 by T_a T_b = (T_{a+b} + T_{b-a}) / 2.
        // result() removes the sign; cheb_moments_from_products() then gives C_k.
        u64 v[M + 1];
        v[0] = seed;
        v[1] = t;
        const u64 t2 = add2(t, t);
        const u64 nt2 = mul2(t, pk2(-2.0f, -2.0f));
#pragma unroll
        for (int k = 2; k <= M; ++k) v[k] = fma2((k & 1) ? t2 : nt2, v[k - 1], v[k - 2]);
        acc[2 * M] = FIRST ? y : add2(acc[2 * M], y);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            acc[k - 1] = FIRST ? v[k] : add2(acc[k - 1], v[k]);
            acc[2 * M + k] = FIRST ? mul2(v[k], y) : fma2(v[k], y, acc[2 * M + k]);
        }
#pragma unroll
        for (int k = M + 1; k <= 2 * M; ++k) {
            const int a = k / 2, b = k - k / 2;
            acc[k - 1] = FIRST ? mul2(v[a], v[b]) : fma2(v[a], v[b], acc[k - 1]);
        }
    }

    // Monomial basis: the powers t^1..t^M by a running product feed S_1..S_M and
    // T_0..T_M; each higher sum S_k, k = M+1..2M, takes the product t^a t^b
    // (a = k/2, b = k - a <= M) in one fma, with as many roundings as the
    // running product would give t^k (2k - 1 in both) and M fewer instructions.
    template <bool FIRST>
    __device__ __forceinline__ void add_pair_powers(u64 t, u64 y) {
        u64 pw[M + 1];
        pw[1] = t;
#pragma unroll
        for (int k = 2; k <= M; ++k) pw[k] = mul2(pw[k - 1], t);
        acc[2 * M] = FIRST ? y : add2(acc[2 * M], y);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            acc[k - 1] = FIRST ? pw[k] : add2(acc[k - 1], pw[k]);
            acc[2 * M + k] = FIRST ? mul2(pw[k], y) : fma2(pw[k], y, acc[2 * M + k]);
        }
#pragma unroll
        for (int k = M + 1; k <= 2 * M; ++k) {
            const int a = k / 2, b = k - k / 2;
            acc[k - 1] = FIRST ? mul2(pw[a], pw[b]) : fma2(pw[a], pw[b], acc[k - 1]);
        }
    }

    // Compensated mode: move the batch sums into the (hi, lo) pairs.
    __device__ __forceinline__ void fold() {
        if (COMP && !SHL) {
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const u64 b = acc[a];
                const u64 s = add2(phi[a], b);
                const u64 bb = sub2(s, phi[a]);
                const u64 e = add2(sub2(phi[a], sub2(s, bb)), sub2(b, bb));
                plo[a] = add2(plo[a], e);
                phi[a] = s;
            }
        }
        if (COMP && SHL) {
#pragma unroll
            for (int a = 0; a < N; ++a) {
                float x0, x1, sh, e;
                up2(acc[a], x0, x1);
                two_sum(shi[a], __fadd_rn(x0, x1), sh, e);
                shi[a] = sh;
                slo[a] = __fadd_rn(slo[a], e);
            }
        }
    }
    // As fold(), and restart the batch at zero (batches fed with add_pair<false>).
    __device__ __forceinline__ void fold_reset() {
        if (COMP) {
            fold();
#pragma unroll
            for (int a = 0; a < N; ++a) acc[a] = 0ull;
        }
    }

    // Chebyshev sign of accumulator a: slot a < 2M holds the moment of
    // degree a + 1 (for a degree k > M the product sum of v_a v_b, sign
    // sigma_a sigma_b), slot 2M + k the right-hand side of degree k.
    static __device__ __forceinline__ bool negated(int a) {
        const int k = a < 2 * M ? a + 1 : a - 2 * M;
        if (CHEB && a < 2 * M && k > M) return ((k / 2) & 2) != ((k - k / 2) & 2);
        return CHEB && (k & 2);
    }

    // Final per-thread value of accumulator a as double-float.
    __device__ __forceinline__ dflt result(int a) const {
        dflt r = result_signed(a);
        if (negated(a)) {
            r.hi = -r.hi;
            r.lo = -r.lo;
        }
        return r;
    }
    __device__ __forceinline__ dflt result_signed(int a) const {
        dflt r;
        if (COMP && !SHL) {
            float x0, x1, l0, l1;
            up2(phi[a], x0, x1);
            up2(plo[a], l0, l1);
            const dflt u = {x0, l0}, v = {x1, l1};
            r = df_add(u, v);
        } else if (COMP) {
            r.hi = shi[a];
            r.lo = slo[a];
        } else {
            float x0, x1;
            up2(acc[a], x0, x1);
            two_sum(x0, x1, r.hi, r.lo);
        }
        return r;
    }
};

// FP64 accumulator (CHEB: Chebyshev basis values, as AccF32).
template <int M, bool CHEB = false>
struct AccF64 {
    static constexpr int N = 3 * M + 1;
    double acc[N];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int a = 0; a < N; ++a) acc[a] = 0.0;
    }
    // Basis values phi_1..phi_M (powers, or T_k by the recurrence) feed the
    // sums of degree 1..M; the slot of degree k = M+1..2M takes phi_a phi_b
    // (a = k/2, b = k - a): the power t^k itself, or for the Chebyshev basis
    // (C_k + C_{b-a}) / 2, turned into C_k by cheb_moments_from_products().
    __device__ __forceinline__ void add_point(double t, double y) {
        double v[M + 1];
        v[0] = 1.0;
        v[1] = t;
#pragma unroll
        for (int k = 2; k <= M; ++k) v[k] = CHEB ? fma(t + t, v[k - 1], -v[k - 2]) : v[k - 1] * t;
        acc[2 * M] += y;
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            acc[k - 1] += v[k];
            acc[2 * M + k] = fma(v[k], y, acc[2 * M + k]);
        }
#pragma unroll
        for (int k = M + 1; k <= 2 * M; ++k) acc[k - 1] = fma(v[k / 2], v[k - k / 2], acc[k - 1]);
    }
};

// ---------------------------------------------------------------------------
// Reductions.  Values are reduced in a fixed order (the result depends only
// on the launch shape, never on timing).
// ---------------------------------------------------------------------------
__device__ __forceinline__ dflt warp_reduce_df(dflt v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
    return v;
}
__device__ __forceinline__ double warp_reduce_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block reduction of N double-float accumulators held per thread; writes the
// N block totals (as doubles) to out[] (shared or global), visible to all
// threads after return.  `red` is shared scratch of kGroup * BLOCK dflt.
// Groups of kGroup accumulators are transposed through shared memory: warp w
// sums accumulator w of the group over all threads (strided, then a warp tree).
template <int BLOCK, int N, typename GetF>
__device__ __forceinline__ void block_reduce_df(GetF get, dflt* red, double* out) {
    constexpr int kWarps = BLOCK / 32;
    constexpr int kGroup = kWarps;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int g0 = 0; g0 < N; g0 += kGroup) {
#pragma unroll
        for (int j = 0; j < kGroup; ++j)
            if (g0 + j < N) red[j * BLOCK + tid] = get(g0 + j);
        __syncthreads();
        if (g0 + warp < N) {
            dflt v = red[warp * BLOCK + lane];
#pragma unroll
            for (int i = 1; i < BLOCK / 32; ++i) v = df_add(v, red[warp * BLOCK + lane + 32 * i]);
            v = warp_reduce_df(v);
            if (lane == 0) out[g0 + warp] = df_to_double(v);
        }
        __syncthreads();
    }
}

// As block_reduce_df, but the block totals stay double-float (no FP64
// instruction: on GB300 FP64 runs at 1/64 of the FP32 rate).
template <int BLOCK, int N, typename GetF>
__device__ __forceinline__ void block_reduce_df2(GetF get, dflt* red, dflt* out) {
    constexpr int kWarps = BLOCK / 32;
    constexpr int kGroup = kWarps;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int g0 = 0; g0 < N; g0 += kGroup) {
#pragma unroll
        for (int j = 0; j < kGroup; ++j)
            if (g0 + j < N) red[j * BLOCK + tid] = get(g0 + j);
        __syncthreads();
        if (g0 + warp < N) {
            dflt v = red[warp * BLOCK + lane];
#pragma unroll
            for (int i = 1; i < BLOCK / 32; ++i) v = df_add(v, red[warp * BLOCK + lane + 32 * i]);
            v = warp_reduce_df(v);
            if (lane == 0) out[g0 + warp] = v;
        }
        __syncthreads();
    }
}

// Warp reduce-scatter by recursive halving: v[0..NP) per lane (entries at
// or beyond the caller's count are zero); on return lane l holds the warp
// total of entry (l mod NP).  At the level of half-size H each lane keeps
// the half of its entries picked by lane bit H and receives the partner's
// copy of that half, so NP-1 exchanges replace the NP*5 of a butterfly per
// entry.  NP is 16 or 32.
template <int NP>
__device__ __forceinline__ dflt warp_reduce_scatter_df(dflt* v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int H = NP / 2; H >= 1; H /= 2) {
        const bool upper = (lane & H) != 0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const dflt keep = upper ? v[H + i] : v[i];
            const dflt send = upper ? v[i] : v[H + i];
            v[i] = df_add(keep, df_shfl_xor(send, H));
        }
    }
#pragma unroll
    for (int o = NP; o < 32; o *= 2) v[0] = df_add(v[0], df_shfl_xor(v[0], o));
    return v[0];
}

template <int NP>
__device__ __forceinline__ double warp_reduce_scatter_d(double* v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int H = NP / 2; H >= 1; H /= 2) {
        const bool upper = (lane & H) != 0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const double keep = upper ? v[H + i] : v[i];
            const double send = upper ? v[i] : v[H + i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, H);
        }
    }
#pragma unroll
    for (int o = NP; o < 32; o *= 2) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    return v[0];
}

template <int BLOCK, int N, typename GetF>
__device__ __forceinline__ void block_reduce_d(GetF get, double* red, double* out) {
    constexpr int kWarps = BLOCK / 32;
    constexpr int kGroup = kWarps;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int g0 = 0; g0 < N; g0 += kGroup) {
#pragma unroll
        for (int j = 0; j < kGroup; ++j)
            if (g0 + j < N) red[j * BLOCK + tid] = get(g0 + j);
        __syncthreads();
        if (g0 + warp < N) {
            double v = red[warp * BLOCK + lane];
#pragma unroll
            for (int i = 1; i < BLOCK / 32; ++i) v += red[warp * BLOCK + lane + 32 * i];
            v = warp_reduce_d(v);
            if (lane == 0) out[g0 + warp] = v;
        }
        __syncthreads();
    }
}

// Chebyshev moments C_k = sum T_k(t) of degree k = m+1..2m from the product
// sums P_k = sum T_a(t) T_b(t), a = k/2, b = k - a, that the accumulators keep
// for those degrees: T_a T_b = (T_k + T_{b-a}) / 2 gives C_k = 2 P_k - C_{b-a},
// with b - a = 0 (C_0: the point count, or the weight sum) or 1.  mo[0..2m]
// holds C_0, the moments up to degree m and the product sums above.
__host__ __device__ __forceinline__ void cheb_moments_from_products(int m, double* mo) {
    for (int k = m + 1; k <= 2 * m; ++k) mo[k] = 2.0 * mo[k] - mo[(k - k / 2) - k / 2];
}

// ---------------------------------------------------------------------------
// FP64 solve of the Hankel normal system (Section II) of runtime degree
// m <= NMAX.  S = S_0..S_2m, T = T_0..T_m.  The (m+1)x(m+1) system is
// embedded in an (NMAX+1)-square one as [[A, 0], [0, I]] so that lanes of a
// warp solving systems of different degrees run the same instructions; the
// padding changes no arithmetic on the real block (its entries only ever
// meet zeros).  Partial pivoting takes the first row of largest magnitude;
// a pivot at or below (m+1) * eps * max|A| is singular (eps: singular_eps).  Writes ncoef
// values of Xt (t basis, may be null) and X (x basis, by expanding
// (s (x - c))^k): m+1 coefficients then zeros.  Returns an LSEFIT status;
// on failure the m+1 coefficients are NaN.
// ---------------------------------------------------------------------------
// Machine epsilon of the arithmetic that formed the power sums: a pivot at
// or below (m+1) * eps * max|A| is treated as zero.  FP32 per-point powers
// alone leave pivots of relative size ~2^-24 in a rank-deficient system.
__host__ __device__ constexpr double singular_eps(int accum) {
    return accum == LSEFIT_ACCUM_F64 ? 2.220446049250313e-16 : 1.1920928955078125e-07;
}

// Comparisons of FP64 values on the integer pipe (an FP64 instruction costs
// ~78 cycles per warp on this part, an integer one ~2): the bit pattern of |v|
// orders like |v| for every non-NaN double, and v is finite exactly when that
// pattern is below the one of infinity.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool finite_bits(double v) {
    return abs_bits(v) < 0x7ff0000000000000ull;
}
// max(acc, |v|) for finite v as bit patterns (acc starts at 0, i.e. +0.0)
__device__ __forceinline__ unsigned long long max_abs_bits(unsigned long long acc, double v) {
    const unsigned long long b = abs_bits(v);
    return b > acc ? b : acc;
}

// 1/a for the eliminations: Newton-Raphson refinement of an approximate
// reciprocal (r <- r + r (1 - a r), each step squaring the relative error;
// see e.g. Muller et al., Handbook of Floating-Point Arithmetic, on Newton
// iterations for the reciprocal).  The seed is the FP32 hardware
// approximation for a's significand m in [1, 2), about 2^-22 relative; two
// steps (four FP64 fmas) bring it to the rounding level of FP64 (within an
// ulp or two; not always correctly rounded).  The exponent goes back by
// integer arithmetic.  On GB300 an FP64 instruction costs a warp about 64
// cycles, FP32 instructions and conversions one or two, so this takes about
// two thirds of the time of IEEE division.  Zero, subnormal, infinite and NaN
// pivots and |a| >= 2^1022 (met only by singular or overflowing systems)
// take IEEE division.
__device__ __forceinline__ double recip_f64(double a) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    const int ex = (int)((bits >> 52) & 0x7ffu);
    if (ex == 0 || ex > 2044) return 1.0 / a;
    const double m = __longlong_as_double((long long)((bits & 0x800fffffffffffffull) | 0x3ff0000000000000ull));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__double2float_rn(m)));
    double r = (double)rf;
    double e = fma(-m, r, 1.0);
    r = fma(r, e, r);
    e = fma(-m, r, 1.0);
    r = fma(r, e, r);
    // 1/a = r 2^(1023 - ex), r in [0.5, 1]: shift r's exponent field
    return __longlong_as_double(__double_as_longlong(r) + ((long long)(1023 - ex) << 52));
}

// Gaussian elimination with partial pivoting of the padded system A z = r
// (A[.][N] holds r; rows and columns beyond m are the identity), then back
// substitution.  The pivot is the first row of largest |a_rk|; a pivot of a
// row <= m at or below tol is singular.  Returns LSEFIT_OK or
// LSEFIT_ERR_SINGULAR; z[0..m] is the solution.
template <int NMAX>
__device__ __forceinline__ int ge_padded(int m, double (&A)[NMAX + 1][NMAX + 2], double tol, double* z) {
    constexpr int N = NMAX + 1;
    int st = LSEFIT_OK;
    double inv_piv[N];  // reciprocal of each pivot, reused by the back-substitution
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int p = k;
        unsigned long long best = abs_bits(A[k][k]);
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            const unsigned long long v = abs_bits(A[r][k]);
            if (v > best) {
                best = v;
                p = r;
            }
        }
        // best <= tol, compared on the integer pipe (tol is finite and >= 0)
        if (k <= m && !(best > (unsigned long long)__double_as_longlong(tol))) st = LSEFIT_ERR_SINGULAR;
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            if (r == p) {
#pragma unroll
                for (int j = k; j <= N; ++j) {
                    const double tmp = A[k][j];
                    A[k][j] = A[r][j];
                    A[r][j] = tmp;
                }
            }
        }
        const double inv = recip_f64(A[k][k]);
        inv_piv[k] = inv;
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            const double f = A[r][k] * inv;
#pragma unroll
            for (int j = k + 1; j <= N; ++j) A[r][j] = fma(-f, A[k][j], A[r][j]);
        }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        double acc = A[i][N];
#pragma unroll
        for (int j = i + 1; j < N; ++j) acc = fma(-A[i][j], z[j], acc);
        z[i] = acc * inv_piv[i];
    }
    if (st == LSEFIT_OK) {
        bool zf = true;
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i <= m) zf = zf && finite_bits(z[i]);
        if (!zf) st = LSEFIT_ERR_SINGULAR;
    }
    return st;
}

template <int NMAX>
__device__ __forceinline__ int hankel_ge(int m, const double* S, const double* rhs, double* z, double eps) {
    constexpr int N = NMAX + 1;
    double A[N][N + 1];
    // max|A| over the 2m+1 distinct entries S_0..S_2m of the Hankel matrix
    // (finite: checked before the elimination)
    unsigned long long ab = 0ull;
#pragma unroll
    for (int k = 0; k <= 2 * NMAX; ++k)
        if (k <= 2 * m) ab = max_abs_bits(ab, S[k]);
    const double amax = __longlong_as_double((long long)ab);
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int k = 0; k < N; ++k) A[j][k] = (j <= m && k <= m) ? S[j + k] : ((j == k) ? 1.0 : 0.0);
        A[j][N] = (j <= m) ? rhs[j] : 0.0;
    }
    return ge_padded<NMAX>(m, A, (double)(m + 1) * eps * amax, z);
}

// Cholesky factorisation of the padded system (the Hankel matrix is
// symmetric positive definite for distinct abscissae): A = L L^T, then
// L w = rhs and L^T z = w.  A diagonal pivot at or below (m+1) * eps * max|A|
// is singular.  The padded identity block factors to itself.
template <int NMAX>
__device__ __forceinline__ int hankel_cholesky(int m, const double* S, const double* rhs, double* z, double eps) {
    constexpr int N = NMAX + 1;
    unsigned long long ab = 0ull;
#pragma unroll
    for (int k = 0; k <= 2 * NMAX; ++k)
        if (k <= 2 * m) ab = max_abs_bits(ab, S[k]);
    const double tol = (double)(m + 1) * eps * __longlong_as_double((long long)ab);
    double Lm[N][N];
    double inv[N];
    int st = LSEFIT_OK;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        double d = (j <= m) ? S[2 * j] : 1.0;
#pragma unroll
        for (int k = 0; k < j; ++k) d = fma(-Lm[j][k], Lm[j][k], d);
        if (j <= m && !(d > tol)) st = LSEFIT_ERR_SINGULAR;
        const double ljj = sqrt(fmax(d, 0.0));
        Lm[j][j] = ljj;
        inv[j] = recip_f64(ljj);
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            double v = (i <= m && j <= m) ? S[i + j] : 0.0;
#pragma unroll
            for (int k = 0; k < j; ++k) v = fma(-Lm[i][k], Lm[j][k], v);
            Lm[i][j] = v * inv[j];
        }
    }
    double w[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double acc = (i <= m) ? rhs[i] : 0.0;
#pragma unroll
        for (int k = 0; k < i; ++k) acc = fma(-Lm[i][k], w[k], acc);
        w[i] = acc * inv[i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        double acc = w[i];
#pragma unroll
        for (int k = i + 1; k < N; ++k) acc = fma(-Lm[k][i], z[k], acc);
        z[i] = acc * inv[i];
    }
    if (st == LSEFIT_OK) {
        bool zf = true;
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i <= m) zf = zf && finite_bits(z[i]);
        if (!zf) st = LSEFIT_ERR_SINGULAR;
    }
    return st;
}

// Checks that precede the elimination: interval, point count, finiteness
// (m <= NMAX; the loads of S and T are issued together).
template <int NMAX>
__device__ __forceinline__ int fit_precheck(int m, const double* S, const double* T, bool map_ok) {
    if (!map_ok) return LSEFIT_ERR_BAD_INTERVAL;
    if (!(S[0] >= (double)(m + 1))) return LSEFIT_ERR_N_TOO_SMALL;
    bool fin = true;
#pragma unroll
    for (int k = 0; k <= 2 * NMAX; ++k)
        if (k <= 2 * m) fin = fin & finite_bits(S[k]);
#pragma unroll
    for (int k = 0; k <= NMAX; ++k)
        if (k <= m) fin = fin & finite_bits(T[k]);
    return fin ? LSEFIT_OK : LSEFIT_ERR_NONFINITE;
}

// Un-map of t-basis coefficients z (k <= m) to the monomials of x, i.e. the
// coefficients of f(x) = sum_k z_k (s (x - c))^k:  first r_k = z_k s^k (the
// polynomial in u = x - c), then a Taylor shift by -c -- m passes of
// synthetic division, r_j <- r_j - c r_{j+1} for j = m-1 down to i -- which
// expands sum_k r_k (x - c)^k.  (m(m+1)/2 + 2m FP64 operations, where the
// binomial expansion out_j = sum_{k>=j} z_k C(k,j) s^k (-c)^(k-j) takes about
// 2(m+1)^2 + m(m+1)/2.)
template <int NMAX>
__device__ __forceinline__ void unmap_padded(int m, const double* z, double c, double s, double* out) {
    constexpr int N = NMAX + 1;
    double sk = 1.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        out[k] = (k <= m) ? z[k] * sk : 0.0;
        if (k < m) sk *= s;
    }
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
#pragma unroll
        for (int j = N - 2; j >= i; --j)
            if (i < m && j < m) out[j] = fma(-c, out[j + 1], out[j]);
    }
}

// identity: the caller knows c = 0 and s = 1 (the un-map is then the identity
// exactly, and is skipped).
template <int NMAX, bool CHOL = false>
__device__ int solve_hankel_rt(int m, const double* S, const double* T, double c, double s,
                               bool map_ok, double eps, double* Xt, double* X, int ncoef, bool identity = false) {
    constexpr int N = NMAX + 1;
    double z[N];
    int st = fit_precheck<NMAX>(m, S, T, map_ok);
    if (st == LSEFIT_OK) st = CHOL ? hankel_cholesky<NMAX>(m, S, T, z, eps) : hankel_ge<NMAX>(m, S, T, z, eps);
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    if (st != LSEFIT_OK) {
        for (int i = 0; i < ncoef; ++i) {
            const double v = i <= m ? qnan : 0.0;
            if (Xt) Xt[i] = v;
            X[i] = v;
        }
        return st;
    }
    double out[N];
    if (identity) {
#pragma unroll
        for (int j = 0; j < N; ++j) out[j] = z[j];
    } else {
        unmap_padded<NMAX>(m, z, c, s, out);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < ncoef) {
            if (Xt) Xt[i] = i <= m ? z[i] : 0.0;
            X[i] = i <= m ? out[i] : 0.0;
        }
    }
    for (int i = N; i < ncoef; ++i) {
        if (Xt) Xt[i] = 0.0;
        X[i] = 0.0;
    }
    return LSEFIT_OK;
}

// Monomial coefficients of sum_k a_k T_k(t) (k <= m): the recurrence of the
// basis applied to coefficient rows, P_{k+1}(t) = 2 t P_k(t) - P_{k-1}(t).
template <int NMAX>
__device__ __forceinline__ void cheb_to_mono(int m, const double* a, double* out) {
    constexpr int N = NMAX + 1;
    double pm1[N], p[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        pm1[j] = j == 0 ? 1.0 : 0.0;
        p[j] = j == 1 ? 1.0 : 0.0;
        out[j] = a[0] * pm1[j] + (m >= 1 ? a[1] * p[j] : 0.0);
    }
#pragma unroll
    for (int k = 2; k < N; ++k) {
        if (k > m) break;
#pragma unroll
        for (int j = N - 1; j >= 0; --j) {
            const double nj = (j > 0 ? 2.0 * p[j - 1] : 0.0) - pm1[j];
            pm1[j] = p[j];
            p[j] = nj;
            out[j] = fma(a[k], nj, out[j]);
        }
    }
}

// Solve of the generalised normal equations from the moments Mo[0..2m] and
// right-hand sides T[0..m] (count = number of points).  Monomial basis:
// G[j][k] = Mo[j+k]; Chebyshev: G[j][k] = (Mo[j+k] + Mo[|j-k|]) / 2.
// Singular when a pivot is at or below (m+1) * eps * max|G|.  Writes Xb (the
// coefficients in the basis of t) and X (monomials of x), NaN on failure.
template <int NMAX, bool CHEB>
__device__ int solve_general_rt(int m, const double* Mo, const double* T, double count, double c, double s,
                                bool map_ok, double eps, double* Xb, double* X, int ncoef) {
    constexpr int N = NMAX + 1;
    int st = LSEFIT_OK;
    if (!map_ok) st = LSEFIT_ERR_BAD_INTERVAL;
    else if (!(count >= (double)(m + 1))) st = LSEFIT_ERR_N_TOO_SMALL;
    if (st == LSEFIT_OK) {
        bool fin = true;
#pragma unroll
        for (int k = 0; k <= 2 * NMAX; ++k)
            if (k <= 2 * m) fin = fin & finite_bits(Mo[k]);
#pragma unroll
        for (int k = 0; k <= NMAX; ++k)
            if (k <= m) fin = fin & finite_bits(T[k]);
        if (!fin) st = LSEFIT_ERR_NONFINITE;
    }
    double z[N];
    if (st == LSEFIT_OK) {
        double A[N][N + 1];
        unsigned long long ab = 0ull;
#pragma unroll
        for (int j = 0; j < N; ++j) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                double g = (j == k) ? 1.0 : 0.0;
                if (j <= m && k <= m) {
                    g = CHEB ? 0.5 * (Mo[j + k] + Mo[j > k ? j - k : k - j]) : Mo[j + k];
                    ab = max_abs_bits(ab, g);
                }
                A[j][k] = g;
            }
            A[j][N] = (j <= m) ? T[j] : 0.0;
        }
        st = ge_padded<NMAX>(m, A, (double)(m + 1) * eps * __longlong_as_double((long long)ab), z);
    }
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    if (st != LSEFIT_OK) {
        for (int i = 0; i < ncoef; ++i) {
            const double v = i <= m ? qnan : 0.0;
            if (Xb) Xb[i] = v;
            X[i] = v;
        }
        return st;
    }
    double zt[N], out[N];
    if (CHEB) {
        cheb_to_mono<NMAX>(m, z, zt);
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j) zt[j] = z[j];
    }
    unmap_padded<NMAX>(m, zt, c, s, out);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < ncoef) {
            if (Xb) Xb[i] = i <= m ? z[i] : 0.0;
            X[i] = i <= m ? out[i] : 0.0;
        }
    }
    for (int i = N; i < ncoef; ++i) {
        if (Xb) Xb[i] = 0.0;
        X[i] = 0.0;
    }
    return LSEFIT_OK;
}

// ---------------------------------------------------------------------------
// Accumulation of the points of one contiguous range [b, e) by `nthreads`
// cooperating threads (`rank` = this thread's index among them): 16-byte
// vectors of x and y when both start at the same offset within 16 bytes,
// scalar loads for the unaligned head, the tail, and the rest otherwise.
// ---------------------------------------------------------------------------
template <int DT>
__device__ __forceinline__ void split_range(const void* x, const void* y, int64_t b, int64_t e,
                                            int64_t& head, int64_t& nvec) {
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec;
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x) + (uintptr_t)b * ES;
    const uintptr_t ya = reinterpret_cast<uintptr_t>(y) + (uintptr_t)b * ES;
    const int64_t len = e - b;
    if ((xa & 15) == (ya & 15) && (xa % ES) == 0) {
        int64_t h = (int64_t)(((16 - (xa & 15)) & 15) / ES);
        head = h < len ? h : len;
        nvec = (len - head) / PV;
    } else {
        head = len;
        nvec = 0;
    }
}

// Unpack one 16-byte vector of x and of y into packed pairs and feed them.
template <int M, int DT, bool COMP, bool MAP, bool FIRST, bool SHL = false, bool CHEB = false>
__device__ __forceinline__ void feed_vec(AccF32<M, COMP, SHL, CHEB>& A, uint4 xv, uint4 yv, u64 c2, u64 s2) {
    const u64 one2 = CHEB ? pk2(1.0f, 1.0f) : 0ull;
    if (DT == LSEFIT_F32) {
        u64 xa = pk2(__uint_as_float(xv.x), __uint_as_float(xv.y));
        u64 xb = pk2(__uint_as_float(xv.z), __uint_as_float(xv.w));
        u64 ya = pk2(__uint_as_float(yv.x), __uint_as_float(yv.y));
        u64 yb = pk2(__uint_as_float(yv.z), __uint_as_float(yv.w));
        if (MAP) {
            xa = mul2(sub2(xa, c2), s2);
            xb = mul2(sub2(xb, c2), s2);
        }
        A.template add_pair<FIRST>(xa, ya, one2);
        A.template add_pair<false>(xb, yb, one2);
    } else {  // BF16: 8 points per vector
        const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
        const uint32_t yw[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            u64 xp = pk2(bf16_lo(xw[q]), bf16_hi(xw[q]));
            u64 yp = pk2(bf16_lo(yw[q]), bf16_hi(yw[q]));
            if (MAP) xp = mul2(sub2(xp, c2), s2);
            if (q == 0) A.template add_pair<FIRST>(xp, yp, one2);
            else A.template add_pair<false>(xp, yp, one2);
        }
    }
}

// Groups of UNROLL vectors per compensated batch.  A batch gives each packed
// lane 8 points (16 at degree >= 7, where the fold of 3m+1 slots would
// otherwise be a large share of the per-point work); the naive FP32 sum of a
// batch is the only uncompensated rounding, about (points - 1) ulp of the
// batch's absolute sum.
template <bool COMP, int M, int UNROLL, int PV>
__host__ __device__ constexpr int comp_groups() {
    const int batch = M >= 7 ? 16 : 8;        // points per packed lane
    const int per_group = UNROLL * (PV / 2);  // points per packed lane in one group
    return (!COMP || batch <= per_group) ? 1 : batch / per_group;
}

// Minimum resident blocks of 256 threads for the single-series FP32 passes:
// two up to degree 5 (at most 128 registers, 16 warps per SM), one above,
// where the compensated slots need more registers than two blocks leave.
template <int M>
__host__ __device__ constexpr int pass_min_blocks() {
    return M <= 5 ? 2 : 1;
}

// FP32/BF16 storage, FP32 arithmetic.  In compensated mode each thread's
// batch (comp_groups() x UNROLL vectors, or one scalar point) is folded into
// its TwoSum pairs.
template <int M, int DT, bool COMP, bool MAP, int UNROLL, bool SHL = false, bool CHEB = false>
__device__ __forceinline__ void accumulate_range(AccF32<M, COMP, SHL, CHEB>& A, const void* x, const void* y,
                                                 int64_t b, int64_t e, int64_t rank, int64_t nthreads,
                                                 float cf, float sf) {
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec;
    int64_t head, nvec;
    split_range<DT>(x, y, b, e, head, nvec);
    const u64 c2 = pk2(cf, cf), s2 = pk2(sf, sf);
    const uint4* xv = reinterpret_cast<const uint4*>(static_cast<const char*>(x) + (b + head) * ES);
    const uint4* yv = reinterpret_cast<const uint4*>(static_cast<const char*>(y) + (b + head) * ES);
    int64_t v = rank;
    constexpr int G = comp_groups<COMP, M, UNROLL, PV>();
    for (; v + (G * UNROLL - 1) * nthreads < nvec; v += G * UNROLL * nthreads) {
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
            uint4 xr[UNROLL], yr[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                xr[u] = ld_stream16(xv + v + (gi * UNROLL + u) * nthreads);
                yr[u] = ld_stream16(yv + v + (gi * UNROLL + u) * nthreads);
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (gi == 0 && u == 0) feed_vec<M, DT, COMP, MAP, COMP, SHL, CHEB>(A, xr[u], yr[u], c2, s2);
                else feed_vec<M, DT, COMP, MAP, false, SHL, CHEB>(A, xr[u], yr[u], c2, s2);
            }
        }
        A.fold();
    }
    for (; v < nvec; v += nthreads) {
        feed_vec<M, DT, COMP, MAP, COMP, SHL, CHEB>(A, ld_stream16(xv + v), ld_stream16(yv + v), c2, s2);
        A.fold();
    }
    // scalar points: [b, b + head) and [b + head + nvec * PV, e)
    const int64_t tail0 = b + head + nvec * PV;
    const int64_t nscalar = head + (e - tail0);
    for (int64_t q = rank; q < nscalar; q += nthreads) {
        const int64_t i = q < head ? b + q : tail0 + (q - head);
        float xs = Elem<DT>::ld(x, i);
        const float ys = Elem<DT>::ld(y, i);
        if (MAP) xs = __fmul_rn(__fsub_rn(xs, cf), sf);
        A.template add_pair<COMP>(pk2(xs, 0.0f), pk2(ys, 0.0f), pk2(1.0f, 0.0f));
        A.fold();
    }
}

// FP64 arithmetic for any storage.
template <int DT, int PV>
__device__ __forceinline__ void unpack_f64(uint4 r, double* v) {
    if (DT == LSEFIT_F64) {
        v[0] = __hiloint2double(r.y, r.x);
        v[1] = __hiloint2double(r.w, r.z);
    } else if (DT == LSEFIT_F32) {
        v[0] = __uint_as_float(r.x);
        v[1] = __uint_as_float(r.y);
        v[2] = __uint_as_float(r.z);
        v[3] = __uint_as_float(r.w);
    } else {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[2 * q] = bf16_lo(w[q]);
            v[2 * q + 1] = bf16_hi(w[q]);
        }
    }
}

template <int M, int DT, int UNROLL, bool MAP, bool CHEB = false>
__device__ __forceinline__ void accumulate_range_f64(AccF64<M, CHEB>& A, const void* x, const void* y,
                                                     int64_t b, int64_t e, int64_t rank,
                                                     int64_t nthreads, double c, double s) {
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec;
    int64_t head, nvec;
    split_range<DT>(x, y, b, e, head, nvec);
    const uint4* xv = reinterpret_cast<const uint4*>(static_cast<const char*>(x) + (b + head) * ES);
    const uint4* yv = reinterpret_cast<const uint4*>(static_cast<const char*>(y) + (b + head) * ES);
    auto feed = [&](uint4 xr, uint4 yr) {
        double xs[PV], ys[PV];
        unpack_f64<DT, PV>(xr, xs);
        unpack_f64<DT, PV>(yr, ys);
#pragma unroll
        for (int q = 0; q < PV; ++q) A.add_point(MAP ? s * (xs[q] - c) : xs[q], ys[q]);
    };
    int64_t v = rank;
    for (; v + (UNROLL - 1) * nthreads < nvec; v += UNROLL * nthreads) {
        uint4 xr[UNROLL], yr[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            xr[u] = ld_stream16(xv + v + u * nthreads);
            yr[u] = ld_stream16(yv + v + u * nthreads);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) feed(xr[u], yr[u]);
    }
    for (; v < nvec; v += nthreads) feed(ld_stream16(xv + v), ld_stream16(yv + v));
    const int64_t tail0 = b + head + nvec * PV;
    const int64_t nscalar = head + (e - tail0);
    for (int64_t q = rank; q < nscalar; q += nthreads) {
        const int64_t i = q < head ? b + q : tail0 + (q - head);
        const double xs = Elem<DT>::ld64(x, i);
        A.add_point(MAP ? s * (xs - c) : xs, Elem<DT>::ld64(y, i));
    }
}

// Degree dispatch for runtime m.
template <template <int> class F, typename... Args>
__device__ __forceinline__ auto by_degree(int m, Args... args) {
    switch (m) {
        case 1: return F<1>::run(args...);
        case 2: return F<2>::run(args...);
        case 3: return F<3>::run(args...);
        case 4: return F<4>::run(args...);
        case 5: return F<5>::run(args...);
        case 6: return F<6>::run(args...);
        case 7: return F<7>::run(args...);
        default: return F<8>::run(args...);
    }
}

}  // namespace lsefit
