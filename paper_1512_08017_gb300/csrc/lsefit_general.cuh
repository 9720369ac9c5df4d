// lsefit_general.cuh -- the generalised objective: per-point weights and the
// Chebyshev basis.
//
// Section II minimises sum_i [y_i - f(x_i)]^2 over the monomials of x.  Two
// generalisations keep its single pass and its small dense solve:
//   * weights: sum_i w_i [y_i - f(t_i)]^2.  The normal matrix and right-hand
//     side take a factor w_i in every sum: M_k = sum w t^k, T_k = sum w t^k y;
//   * the Chebyshev basis f(t) = sum_k a_k T_k(t) (T_0 = 1, T_1 = t,
//     T_{k+1} = 2 t T_k - T_{k-1}), which stays well conditioned on [-1, 1]
//     where the monomial Hankel matrix does not.  The product identity
//     T_j T_k = (T_{j+k} + T_{|j-k|}) / 2 makes the normal matrix
//     G[j][k] = (C_{j+k} + C_{|j-k|}) / 2 a function of the 2m+1 moments
//     C_p = sum w T_p(t), so the pass still keeps 3m+1 (+1) accumulators.
// Both run the basis recurrence on w-scaled values: b_0 = w, b_1 = w t, then
// b_{k+1} = 2 t b_k - b_{k-1} (Chebyshev) or b_{k+1} = t b_k (monomial).
// The Chebyshev values are carried as sigma_k b_k with sigma_k = -1 for
// k = 2, 3 (mod 4), +1 otherwise: then sigma_{k+1} sigma_{k-1} = -1 and every
// step is one fma, sigma_{k+1} b_{k+1} = (+-2t) (sigma_k b_k) + sigma_{k-1} b_{k-1},
// with no negation.  Rounding to nearest is symmetric under negation, so the
// sums are the exact negatives of the unsigned ones; result() restores the
// sign.
#pragma once

#include "lsefit_device.cuh"

namespace lsefit {

// Accumulator slots: 0..2M the moments M_k = sum w phi_k(t), 2M+1..3M+1 the
// right-hand sides T_k = sum w phi_k(t) y.  Without weights slot 0 (the
// point count) is not accumulated.  The `w` operand of add_pair is the
// weight pair, or, without weights, 1 for a point and 0 for an empty lane
// (it seeds the Chebyshev recurrence, in which an empty lane with t = 0
// would otherwise give T_2(0) = -1).
// Compensation (COMP): per slot a scalar TwoSum pair (hi, lo); a batch's two
// packed lane sums are added in FP32 (one rounding of the batch's own size)
// and then moved into (hi, lo) exactly.
template <int M, bool COMP, bool W, bool CHEB>
struct AccGenF32 {
    static constexpr int N = 3 * M + 2;
    static constexpr int K0 = W ? 0 : 1;
    u64 acc[N];
    float shi[COMP ? N : 1], slo[COMP ? N : 1];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int a = 0; a < N; ++a) {
            acc[a] = 0ull;
            if (COMP) {
                shi[a] = 0.0f;
                slo[a] = 0.0f;
            }
        }
    }

    template <bool FIRST>
    __device__ __forceinline__ void put(int a, u64 v) {
        acc[a] = FIRST ? v : add2(acc[a], v);
    }
    template <bool FIRST>
    __device__ __forceinline__ void put_fma(int a, u64 b, u64 y) {
        acc[a] = FIRST ? mul2(b, y) : fma2(b, y, acc[a]);
    }

    // Add the two points (t.x, y.x, w.x), (t.y, y.y, w.y).  FIRST assigns
    // instead of adding (the first pair of a compensated batch).
    template <bool FIRST>
    __device__ __forceinline__ void add_pair(u64 t, u64 y, u64 w) {
        if (!W) {
            add_pair_unweighted<FIRST>(t, y, w);
            return;
        }
        if (W) {
            put<FIRST>(0, w);
            put_fma<FIRST>(2 * M + 1, w, y);
        } else {
            put<FIRST>(2 * M + 1, y);
        }
        const u64 b1 = W ? mul2(w, t) : t;
        put<FIRST>(1, b1);
        put_fma<FIRST>(2 * M + 2, b1, y);
        const u64 t2 = CHEB ? add2(t, t) : 0ull;
        const u64 nt2 = CHEB ? mul2(t, pk2(-2.0f, -2.0f)) : 0ull;
        u64 bm2 = w, bm1 = b1;
#pragma unroll
        for (int k = 2; k <= 2 * M; ++k) {
            // sigma_k sigma_{k-1} = -1 for even k, +1 for odd k
            const u64 bk = CHEB ? fma2((k & 1) ? t2 : nt2, bm1, bm2) : mul2(bm1, t);
            put<FIRST>(k, bk);
            if (k <= M) put_fma<FIRST>(2 * M + 1 + k, bk, y);
            bm2 = bm1;
            bm1 = bk;
        }
    }

    // Without weights: the basis values phi_1..phi_M (v_k = sigma_k T_k for
    // the Chebyshev basis, seeded by `seed`, 1 per point and 0 for an empty
    // lane) feed the moments of degree 1..M and the right-hand sides; the slot
    // of degree k = M+1..2M takes v_a v_b (a = k/2, b = k - a): t^k for the
    // monomials, sigma_a sigma_b (C_k + C_{b-a}) / 2 for the Chebyshev basis
    // (result() removes the sign, cheb_moments_from_products() gives C_k).
    template <bool FIRST>
    __device__ __forceinline__ void add_pair_unweighted(u64 t, u64 y, u64 seed) {
        u64 v[M + 1];
        v[0] = seed;
        v[1] = t;
        const u64 t2 = CHEB ? add2(t, t) : 0ull;
        const u64 nt2 = CHEB ? mul2(t, pk2(-2.0f, -2.0f)) : 0ull;
#pragma unroll
        for (int k = 2; k <= M; ++k) v[k] = CHEB ? fma2((k & 1) ? t2 : nt2, v[k - 1], v[k - 2]) : mul2(v[k - 1], t);
        put<FIRST>(2 * M + 1, y);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            put<FIRST>(k, v[k]);
            put_fma<FIRST>(2 * M + 1 + k, v[k], y);
        }
#pragma unroll
        for (int k = M + 1; k <= 2 * M; ++k) put_fma<FIRST>(k, v[k / 2], v[k - k / 2]);
    }

    // Compensated mode: move the batch sums into the (hi, lo) pairs (TwoSum).
    __device__ __forceinline__ void fold() {
        if (COMP) {
#pragma unroll
            for (int a = K0; a < N; ++a) {
                float x0, x1, sh, e;
                up2(acc[a], x0, x1);
                two_sum(shi[a], __fadd_rn(x0, x1), sh, e);
                shi[a] = sh;
                slo[a] = __fadd_rn(slo[a], e);
            }
        }
    }

    // Basis index of slot a (moments 0..2M, then right-hand sides 0..M) and
    // the sign its Chebyshev sums carry.
    static __device__ __forceinline__ bool negated(int a) {
        const int k = a <= 2 * M ? a : a - (2 * M + 1);
        if (CHEB && !W && a <= 2 * M && k > M) return ((k / 2) & 2) != ((k - k / 2) & 2);
        return CHEB && (k & 2);
    }

    // Final per-thread value of slot a as double-float.
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
        if (a < K0) {
            r.hi = 0.0f;
            r.lo = 0.0f;
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

template <int M, bool W, bool CHEB>
struct AccGenF64 {
    static constexpr int N = 3 * M + 2;
    double acc[N];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int a = 0; a < N; ++a) acc[a] = 0.0;
    }
    __device__ __forceinline__ void add_point(double t, double y, double w) {
        if (!W) {
            // as AccGenF32::add_pair_unweighted: products for the degrees above M
            double v[M + 1];
            v[0] = 1.0;
            v[1] = t;
#pragma unroll
            for (int k = 2; k <= M; ++k) v[k] = CHEB ? fma(t + t, v[k - 1], -v[k - 2]) : v[k - 1] * t;
            acc[2 * M + 1] += y;
#pragma unroll
            for (int k = 1; k <= M; ++k) {
                acc[k] += v[k];
                acc[2 * M + 1 + k] = fma(v[k], y, acc[2 * M + 1 + k]);
            }
#pragma unroll
            for (int k = M + 1; k <= 2 * M; ++k) acc[k] = fma(v[k / 2], v[k - k / 2], acc[k]);
            return;
        }
        if (W) {
            acc[0] += w;
            acc[2 * M + 1] = fma(w, y, acc[2 * M + 1]);
        } else {
            acc[2 * M + 1] += y;
        }
        const double b1 = W ? w * t : t;
        acc[1] += b1;
        acc[2 * M + 2] = fma(b1, y, acc[2 * M + 2]);
        const double t2 = t + t;
        double bm2 = W ? w : 1.0, bm1 = b1;
#pragma unroll
        for (int k = 2; k <= 2 * M; ++k) {
            const double bk = CHEB ? fma(t2, bm1, -bm2) : bm1 * t;
            acc[k] += bk;
            if (k <= M) acc[2 * M + 1 + k] = fma(bk, y, acc[2 * M + 1 + k]);
            bm2 = bm1;
            bm1 = bk;
        }
    }
};

// Vectorised split of [b, e) for three streams: 16-byte vectors when x, y
// (and w) start at the same offset within 16 bytes, scalar loads otherwise.
template <int DT, bool W>
__device__ __forceinline__ void split_range3(const void* x, const void* y, const void* w, int64_t b, int64_t e,
                                             int64_t& head, int64_t& nvec) {
    split_range<DT>(x, y, b, e, head, nvec);
    if (W && nvec > 0) {
        int64_t h2, n2;
        split_range<DT>(x, w, b, e, h2, n2);
        if (h2 != head || n2 != nvec) {
            head = e - b;
            nvec = 0;
        }
    }
}

// Grid steps the FP32 general pass prefetches into L2 ahead of its loads
// (degrees up to 4, two blocks per SM): the prefetch of a block's slice of a later
// step holds no registers, and the loads then find their lines in L2.
#ifndef LSEFIT_GEN_PREFETCH_STEPS
#define LSEFIT_GEN_PREFETCH_STEPS 8
#endif
constexpr int kGenPrefetchSteps = LSEFIT_GEN_PREFETCH_STEPS;

// Degrees above 5 (one block per SM): groups of loads ahead of the group
// being fed that each thread prefetches into L2, its own vectors.  Measured
// on the degree-8 Chebyshev passes at 2^28 points: weighted 0.68 of HBM
// without and 0.76 with a prefetch 4 groups ahead; unweighted 0.54 without,
// 0.65-0.66 with it at 384 threads per block (below).
#ifndef LSEFIT_GEN_THREAD_PREFETCH
#define LSEFIT_GEN_THREAD_PREFETCH 4
#endif
constexpr int kGenThreadPrefetch = LSEFIT_GEN_THREAD_PREFETCH;

// FP32 arithmetic (FP32 or BF16 storage) over [b, e), map always applied
// (identity constants when the caller gave no interval).  rank is
// blockIdx.x * blockDim.x + threadIdx.x: a block's threads read consecutive
// vectors at every grid step, the slice thread 0 prefetches.
template <int M, int DT, bool COMP, bool W, bool CHEB, int UNROLL>
__device__ __forceinline__ void accumulate_range_gen(AccGenF32<M, COMP, W, CHEB>& A, const void* x, const void* y,
                                                     const void* w, int64_t b, int64_t e, int64_t rank,
                                                     int64_t nthreads, float cf, float sf) {
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec;
    int64_t head, nvec;
    split_range3<DT, W>(x, y, w, b, e, head, nvec);
    const u64 c2 = pk2(cf, cf), s2 = pk2(sf, sf), one2 = pk2(1.0f, 1.0f);
    const uint4* xv = reinterpret_cast<const uint4*>(static_cast<const char*>(x) + (b + head) * ES);
    const uint4* yv = reinterpret_cast<const uint4*>(static_cast<const char*>(y) + (b + head) * ES);
    const uint4* wv = W ? reinterpret_cast<const uint4*>(static_cast<const char*>(w) + (b + head) * ES) : nullptr;
    auto feed = [&](uint4 xr, uint4 yr, uint4 wr, bool first) {
        const uint32_t xw[4] = {xr.x, xr.y, xr.z, xr.w};
        const uint32_t yw[4] = {yr.x, yr.y, yr.z, yr.w};
        const uint32_t ww[4] = {wr.x, wr.y, wr.z, wr.w};
#pragma unroll
        for (int k = 0; k < PV / 2; ++k) {
            u64 tp, yp, wp = one2;
            if (DT == LSEFIT_F32) {
                tp = pk2(__uint_as_float(xw[2 * k]), __uint_as_float(xw[2 * k + 1]));
                yp = pk2(__uint_as_float(yw[2 * k]), __uint_as_float(yw[2 * k + 1]));
                if (W) wp = pk2(__uint_as_float(ww[2 * k]), __uint_as_float(ww[2 * k + 1]));
            } else {
                tp = pk2(bf16_lo(xw[k]), bf16_hi(xw[k]));
                yp = pk2(bf16_lo(yw[k]), bf16_hi(yw[k]));
                if (W) wp = pk2(bf16_lo(ww[k]), bf16_hi(ww[k]));
            }
            tp = mul2(sub2(tp, c2), s2);
            if (COMP && first && k == 0) A.template add_pair<true>(tp, yp, wp);
            else A.template add_pair<false>(tp, yp, wp);
        }
    };
    constexpr int G = comp_groups<COMP, M, UNROLL, PV>();
    constexpr int GU = G * UNROLL;
    auto load_group = [&](uint4 (&xr)[UNROLL], uint4 (&yr)[UNROLL], uint4 (&wr)[UNROLL], int64_t o) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            xr[u] = ld_stream16(xv + o + u * nthreads);
            yr[u] = ld_stream16(yv + o + u * nthreads);
            wr[u] = W ? ld_stream16(wv + o + u * nthreads) : make_uint4(0, 0, 0, 0);
        }
    };
    int64_t v = rank;
    // L2 prefetch ahead of the loads.  Up to degree 4 (two blocks per SM)
    // thread 0 prefetches the block's slice of the grid step kGenPrefetchSteps
    // ahead (degree 5 has no registers to spare for it); above degree 5 (one
    // block per SM) each thread prefetches its own vectors kGenThreadPrefetch
    // groups ahead.
    const int64_t blk0 = rank - threadIdx.x;  // slice of step k: [blk0 + k nthreads, + blockDim.x)
    auto prefetch_step = [&](int64_t k) {
        const int64_t v0 = blk0 + k * nthreads;
        if (v0 >= nvec) return;
        const unsigned bytes = (unsigned)(min((int64_t)blockDim.x, nvec - v0) * 16);
        prefetch_l2_bulk(xv + v0, bytes);
        prefetch_l2_bulk(yv + v0, bytes);
        if (W) prefetch_l2_bulk(wv + v0, bytes);
    };
    const bool prefetcher = kGenPrefetchSteps > 0 && M <= 4 && threadIdx.x == 0;
    if (prefetcher)
        for (int k = 0; k < kGenPrefetchSteps; ++k) prefetch_step(k);
    int64_t step = 0;  // grid step of this iteration's first load
    for (; v + (GU - 1) * nthreads < nvec; v += GU * nthreads, step += GU) {
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
            uint4 xr[UNROLL], yr[UNROLL], wr[UNROLL];
            if (pass_min_blocks<M>() == 1 && kGenThreadPrefetch > 0) {
                const int64_t po = v + (gi + kGenThreadPrefetch) * UNROLL * nthreads;
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const int64_t q = min(po + u * nthreads, nvec - 1);
                    prefetch_l2(xv + q);
                    prefetch_l2(yv + q);
                    if (W) prefetch_l2(wv + q);
                }
            }
            if (prefetcher)
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) prefetch_step(step + gi * UNROLL + u + kGenPrefetchSteps);
            load_group(xr, yr, wr, v + gi * UNROLL * nthreads);
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) feed(xr[u], yr[u], wr[u], gi == 0 && u == 0);
        }
        A.fold();
    }
    for (; v < nvec; v += nthreads) {
        feed(ld_stream16(xv + v), ld_stream16(yv + v), W ? ld_stream16(wv + v) : make_uint4(0, 0, 0, 0), true);
        A.fold();
    }
    // scalar points: [b, b + head) and [b + head + nvec * PV, e), the second lane empty
    const int64_t tail0 = b + head + nvec * PV;
    const int64_t nscalar = head + (e - tail0);
    for (int64_t q = rank; q < nscalar; q += nthreads) {
        const int64_t i = q < head ? b + q : tail0 + (q - head);
        const float xs = __fmul_rn(__fsub_rn(Elem<DT>::ld(x, i), cf), sf);
        const float ws = W ? Elem<DT>::ld(w, i) : 1.0f;
        A.template add_pair<COMP>(pk2(xs, 0.0f), pk2(Elem<DT>::ld(y, i), 0.0f), pk2(ws, 0.0f));
        A.fold();
    }
}

// FP64 arithmetic for any storage.
template <int M, int DT, bool W, bool CHEB, int UNROLL>
__device__ __forceinline__ void accumulate_range_gen_f64(AccGenF64<M, W, CHEB>& A, const void* x, const void* y,
                                                         const void* w, int64_t b, int64_t e, int64_t rank,
                                                         int64_t nthreads, double c, double s) {
    constexpr int ES = Elem<DT>::kSize, PV = Elem<DT>::kPerVec;
    int64_t head, nvec;
    split_range3<DT, W>(x, y, w, b, e, head, nvec);
    const uint4* xv = reinterpret_cast<const uint4*>(static_cast<const char*>(x) + (b + head) * ES);
    const uint4* yv = reinterpret_cast<const uint4*>(static_cast<const char*>(y) + (b + head) * ES);
    const uint4* wv = W ? reinterpret_cast<const uint4*>(static_cast<const char*>(w) + (b + head) * ES) : nullptr;
    auto feed = [&](uint4 xr, uint4 yr, uint4 wr) {
        double xs[PV], ys[PV], ws[PV];
        unpack_f64<DT, PV>(xr, xs);
        unpack_f64<DT, PV>(yr, ys);
        if (W) unpack_f64<DT, PV>(wr, ws);
#pragma unroll
        for (int q = 0; q < PV; ++q) A.add_point(s * (xs[q] - c), ys[q], W ? ws[q] : 1.0);
    };
    int64_t v = rank;
    for (; v + (UNROLL - 1) * nthreads < nvec; v += UNROLL * nthreads) {
        uint4 xr[UNROLL], yr[UNROLL], wr[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            xr[u] = ld_stream16(xv + v + u * nthreads);
            yr[u] = ld_stream16(yv + v + u * nthreads);
            wr[u] = W ? ld_stream16(wv + v + u * nthreads) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) feed(xr[u], yr[u], wr[u]);
    }
    for (; v < nvec; v += nthreads)
        feed(ld_stream16(xv + v), ld_stream16(yv + v), W ? ld_stream16(wv + v) : make_uint4(0, 0, 0, 0));
    const int64_t tail0 = b + head + nvec * PV;
    const int64_t nscalar = head + (e - tail0);
    for (int64_t q = rank; q < nscalar; q += nthreads) {
        const int64_t i = q < head ? b + q : tail0 + (q - head);
        A.add_point(s * (Elem<DT>::ld64(x, i) - c), Elem<DT>::ld64(y, i), W ? Elem<DT>::ld64(w, i) : 1.0);
    }
}

// ---------------------------------------------------------------------------
// Single-series kernels (as the power-sum pass: per-block partials in FP64,
// the last block combines them in a fixed order and solves).
// ---------------------------------------------------------------------------
constexpr int kGenBlock = 256;
// Threads per block of the pass above degree 5 (one block per SM): at 384 the
// compiler fits the 26 slots of degree 8 in 166-168 registers, 12 warps per
// SM where 256 threads gave 8.  At 2^28 points, Chebyshev m = 8 runs at
// 0.67-0.68 of HBM against 0.61, weighted Chebyshev at 0.78 against 0.75
// (320 threads, whose 10 warps split unevenly over the 4 schedulers: 0.57).
#ifndef LSEFIT_GEN_HI_BLOCK
#define LSEFIT_GEN_HI_BLOCK 384
#endif

struct GenParams {
    const void* x;
    const void* y;
    const void* w;
    int64_t n;
    const double* interval;
    double* sums;           // [3m+2] or null: M_0..M_2m, T_0..T_m
    double* map_out;        // [2] or null
    double* partials;       // [gridDim.x][3m+2]
    unsigned int* ticket;   // zero between calls
    int m_lo;
    double eps;
    double* X;              // [m-m_lo+1][m+1]
    double* Xb;             // same shape or null
    int32_t* status;        // [m-m_lo+1]
};

template <int M, bool W, bool CHEB>
__device__ __noinline__ void gen_solve_degree(const GenParams& p, const double* tot, double c, double s,
                                              bool map_ok, int lane) {
    const int d = p.m_lo + lane;
    p.status[lane] = solve_general_rt<M, CHEB>(d, tot, tot + 2 * M + 1, (double)p.n, c, s, map_ok, p.eps,
                                               p.Xb ? p.Xb + lane * (M + 1) : nullptr, p.X + lane * (M + 1), M + 1);
}

template <int M, bool W, bool CHEB>
__device__ void gen_publish(const GenParams& p, const double* blk, bool map_ok, double c, double s) {
    constexpr int N = 3 * M + 2;
    constexpr int J = kGenBlock / N;
    __shared__ bool s_last;
    __shared__ double comb[kGenBlock];
    __shared__ double tot_s[N];
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
        if (tid == 0 && !W) tot = (double)p.n;
        tot_s[tid] = map_ok ? tot : qnan;
    }
    __syncthreads();
    // without weights, degrees M+1..2M were accumulated as product sums
    if (CHEB && !W && tid == 0) cheb_moments_from_products(M, tot_s);
    __syncthreads();
    if (tid < N && p.sums) p.sums[tid] = tot_s[tid];
    if (tid == 0) {
        if (p.map_out) {
            p.map_out[0] = map_ok ? c : qnan;
            p.map_out[1] = map_ok ? s : qnan;
        }
        *p.ticket = 0u;  // ready for the next call
    }
    __syncthreads();
    if (tid < 32 && tid <= M - p.m_lo) gen_solve_degree<M, W, CHEB>(p, tot_s, c, s, map_ok, tid);
}

template <int M, int DT, bool COMP, bool W, bool CHEB, int UNROLL, int BLOCK = kGenBlock>
__global__ void __launch_bounds__(BLOCK, pass_min_blocks<M>()) gen_kernel_f32(__grid_constant__ const GenParams p) {
    constexpr int N = 3 * M + 2;
    __shared__ dflt red[(BLOCK / 32) * BLOCK];
    __shared__ double blk[N];
    double cd, sd;
    const bool map_ok = map_constants(p.interval, true, cd, sd);
    AccGenF32<M, COMP, W, CHEB> A;
    A.init();
    const int64_t nthr = (int64_t)gridDim.x * BLOCK;
    const int64_t gtid = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
    accumulate_range_gen<M, DT, COMP, W, CHEB, UNROLL>(A, p.x, p.y, p.w, 0, p.n, gtid, nthr, (float)cd, (float)sd);
    block_reduce_df<BLOCK, N>([&](int a) { return A.result(a); }, red, blk);
    gen_publish<M, W, CHEB>(p, blk, map_ok, cd, sd);
}

template <int M, int DT, bool W, bool CHEB, int UNROLL>
__global__ void __launch_bounds__(kGenBlock) gen_kernel_f64(__grid_constant__ const GenParams p) {
    constexpr int N = 3 * M + 2;
    __shared__ double red[(kGenBlock / 32) * kGenBlock];
    __shared__ double blk[N];
    double c, s;
    const bool map_ok = map_constants(p.interval, false, c, s);
    AccGenF64<M, W, CHEB> A;
    A.init();
    const int64_t nthr = (int64_t)gridDim.x * kGenBlock;
    const int64_t gtid = (int64_t)blockIdx.x * kGenBlock + threadIdx.x;
    accumulate_range_gen_f64<M, DT, W, CHEB, UNROLL>(A, p.x, p.y, p.w, 0, p.n, gtid, nthr, c, s);
    block_reduce_d<kGenBlock, N>([&](int a) { return A.acc[a]; }, red, blk);
    gen_publish<M, W, CHEB>(p, blk, map_ok, c, s);
}

typedef void (*gen_kernel_t)(GenParams);

// Kernel for degree M, storage, accumulation and kind.
template <int M, bool W, bool CHEB>
gen_kernel_t gen_pick_m(int dtype, int accum) {
    constexpr int U = W ? 2 : (M <= 4 ? 4 : 2);
    if (accum == LSEFIT_ACCUM_F64) {
        if (dtype == LSEFIT_F64) return gen_kernel_f64<M, LSEFIT_F64, W, CHEB, 2>;
        if (dtype == LSEFIT_F32) return gen_kernel_f64<M, LSEFIT_F32, W, CHEB, 2>;
        return gen_kernel_f64<M, LSEFIT_BF16, W, CHEB, 1>;
    }
    if (dtype == LSEFIT_F64) return nullptr;
    const bool comp = accum == LSEFIT_ACCUM_COMP;
    constexpr int B = pass_min_blocks<M>() == 1 ? LSEFIT_GEN_HI_BLOCK : kGenBlock;
    if (dtype == LSEFIT_F32)
        return comp ? gen_kernel_f32<M, LSEFIT_F32, true, W, CHEB, U, B> : gen_kernel_f32<M, LSEFIT_F32, false, W, CHEB, U, B>;
    return comp ? gen_kernel_f32<M, LSEFIT_BF16, true, W, CHEB, 2, B> : gen_kernel_f32<M, LSEFIT_BF16, false, W, CHEB, 2, B>;
}

template <bool W, bool CHEB>
gen_kernel_t gen_pick(int m, int dtype, int accum) {
    switch (m) {
        case 1: return gen_pick_m<1, W, CHEB>(dtype, accum);
        case 2: return gen_pick_m<2, W, CHEB>(dtype, accum);
        case 3: return gen_pick_m<3, W, CHEB>(dtype, accum);
        case 4: return gen_pick_m<4, W, CHEB>(dtype, accum);
        case 5: return gen_pick_m<5, W, CHEB>(dtype, accum);
        case 6: return gen_pick_m<6, W, CHEB>(dtype, accum);
        case 7: return gen_pick_m<7, W, CHEB>(dtype, accum);
        default: return gen_pick_m<8, W, CHEB>(dtype, accum);
    }
}

// Chebyshev degrees 9..16 (FP64 accumulation only: the compensated FP32 form
// of 3m+2 = 50 slots would need about 300 registers per thread).
template <int M, bool W>
gen_kernel_t gen_pick_high_m(int dtype, int accum) {
    if (accum != LSEFIT_ACCUM_F64) return nullptr;
    if (dtype == LSEFIT_F64) return gen_kernel_f64<M, LSEFIT_F64, W, true, 2>;
    if (dtype == LSEFIT_F32) return gen_kernel_f64<M, LSEFIT_F32, W, true, 2>;
    return gen_kernel_f64<M, LSEFIT_BF16, W, true, 1>;
}

template <bool W>
gen_kernel_t gen_pick_high(int m, int dtype, int accum) {
    switch (m) {
        case 9: return gen_pick_high_m<9, W>(dtype, accum);
        case 10: return gen_pick_high_m<10, W>(dtype, accum);
        case 11: return gen_pick_high_m<11, W>(dtype, accum);
        case 12: return gen_pick_high_m<12, W>(dtype, accum);
        case 13: return gen_pick_high_m<13, W>(dtype, accum);
        case 14: return gen_pick_high_m<14, W>(dtype, accum);
        case 15: return gen_pick_high_m<15, W>(dtype, accum);
        case 16: return gen_pick_high_m<16, W>(dtype, accum);
        default: return nullptr;
    }
}

// One translation unit per kind (and per degree range) instantiates its kernels.
gen_kernel_t gen_pick_weighted(int m, int dtype, int accum);
gen_kernel_t gen_pick_chebyshev(int m, int dtype, int accum);
gen_kernel_t gen_pick_weighted_chebyshev(int m, int dtype, int accum);
gen_kernel_t gen_pick_chebyshev_high(int m, int dtype, int accum);
gen_kernel_t gen_pick_weighted_chebyshev_high(int m, int dtype, int accum);

}  // namespace lsefit
