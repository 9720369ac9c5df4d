/*
 * fit_client.c -- a plain C caller of liblsefit.so (no Python, no torch):
 * allocates device buffers with the CUDA runtime, fits one series with
 * lsefit_fit and a small ragged batch with lsefit_plan_build /
 * lsefit_fit_batched, and prints the coefficients for the test to check.
 *
 * Usage: fit_client <input file> ; the input holds n, then n pairs (x, y),
 * then the batch as S, S+1 offsets and S degrees (points taken from the same
 * x, y arrays).  Output: one line per fit, "status c_0 ... c_m".
 */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lsefit.h"

#define CHECK_CUDA(call)                                                       \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), \
                    __FILE__, __LINE__);                                       \
            return 2;                                                          \
        }                                                                      \
    } while (0)

#define CHECK_LSE(call)                                                        \
    do {                                                                       \
        int r_ = (call);                                                       \
        if (r_ != LSEFIT_OK) {                                                 \
            fprintf(stderr, "lsefit error %s at %s:%d\n",                      \
                    lsefit_status_string(r_), __FILE__, __LINE__);             \
            return 3;                                                          \
        }                                                                      \
    } while (0)

int main(int argc, char** argv) {
    if (argc != 2) return 1;
    FILE* f = fopen(argv[1], "r");
    if (!f) return 1;
    long n = 0;
    if (fscanf(f, "%ld", &n) != 1 || n <= 0) return 1;
    float* hx = (float*)malloc(sizeof(float) * n);
    float* hy = (float*)malloc(sizeof(float) * n);
    for (long i = 0; i < n; ++i)
        if (fscanf(f, "%f %f", &hx[i], &hy[i]) != 2) return 1;
    long S = 0;
    if (fscanf(f, "%ld", &S) != 1 || S <= 0) return 1;
    int64_t* hoff = (int64_t*)malloc(sizeof(int64_t) * (S + 1));
    int32_t* hdeg = (int32_t*)malloc(sizeof(int32_t) * S);
    for (long s = 0; s <= S; ++s) {
        long v;
        if (fscanf(f, "%ld", &v) != 1) return 1;
        hoff[s] = v;
    }
    for (long s = 0; s < S; ++s)
        if (fscanf(f, "%d", &hdeg[s]) != 1) return 1;
    fclose(f);
    if (lsefit_abi_version() != LSEFIT_ABI_VERSION) return 4;

    float *dx, *dy;
    CHECK_CUDA(cudaMalloc((void**)&dx, sizeof(float) * n));
    CHECK_CUDA(cudaMalloc((void**)&dy, sizeof(float) * n));
    CHECK_CUDA(cudaMemcpy(dx, hx, sizeof(float) * n, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(dy, hy, sizeof(float) * n, cudaMemcpyHostToDevice));

    /* one series, degrees 1..3 from one pass, x mapped from [-1, 1] (identity) */
    const int m = 3;
    double interval_h[2] = {-1.0, 1.0};
    double *dinterval, *dX, *dXt;
    int32_t* dst;
    void* ws;
    size_t ws_bytes = lsefit_powersums_workspace_size(m);
    CHECK_CUDA(cudaMalloc((void**)&dinterval, sizeof(interval_h)));
    CHECK_CUDA(cudaMemcpy(dinterval, interval_h, sizeof(interval_h), cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMalloc((void**)&dX, sizeof(double) * 3 * (m + 1)));
    CHECK_CUDA(cudaMalloc((void**)&dXt, sizeof(double) * 3 * (m + 1)));
    CHECK_CUDA(cudaMalloc((void**)&dst, sizeof(int32_t) * 3));
    CHECK_CUDA(cudaMalloc(&ws, ws_bytes));
    CHECK_CUDA(cudaMemset(ws, 0, ws_bytes));
    CHECK_LSE(lsefit_fit(dx, dy, n, LSEFIT_F32, m, 1, LSEFIT_ACCUM_COMP, dinterval, dX, dXt, NULL, NULL, dst, ws,
                         ws_bytes, NULL));
    double hX[3 * (m + 1)];
    int32_t hst[3];
    CHECK_CUDA(cudaMemcpy(hX, dX, sizeof(hX), cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(hst, dst, sizeof(hst), cudaMemcpyDeviceToHost));
    for (int d = 0; d < 3; ++d) {
        printf("single %d %d", d + 1, hst[d]);
        for (int j = 0; j <= m; ++j) printf(" %.17g", hX[d * (m + 1) + j]);
        printf("\n");
    }

    /* the ragged batch */
    int m_max = 1;
    for (long s = 0; s < S; ++s)
        if (hdeg[s] > m_max) m_max = hdeg[s];
    int sms = 0;
    CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    lsefit_plan plan;
    int rc = lsefit_plan_build(hoff, hdeg, S, m_max, NULL, sms, &plan, NULL, 0, NULL, 0);
    if (rc != LSEFIT_OK && rc != LSEFIT_ERR_WORKSPACE) return 3;
    int32_t* hbt = (int32_t*)malloc(sizeof(int32_t) * 4 * (plan.n_block_tasks + 1));
    int32_t* hwt = (int32_t*)malloc(sizeof(int32_t) * 4 * (plan.n_warp_tasks + 1));
    CHECK_LSE(lsefit_plan_build(hoff, hdeg, S, m_max, NULL, sms, &plan, hbt, plan.n_block_tasks, hwt,
                                plan.n_warp_tasks));
    int32_t *dbt, *dwt, *ddeg, *dbst;
    int64_t* doff;
    double *dBX;
    CHECK_CUDA(cudaMalloc((void**)&dbt, sizeof(int32_t) * 4 * (plan.n_block_tasks + 1)));
    CHECK_CUDA(cudaMalloc((void**)&dwt, sizeof(int32_t) * 4 * (plan.n_warp_tasks + 1)));
    CHECK_CUDA(cudaMemcpy(dbt, hbt, sizeof(int32_t) * 4 * plan.n_block_tasks, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(dwt, hwt, sizeof(int32_t) * 4 * plan.n_warp_tasks, cudaMemcpyHostToDevice));
    plan.block_tasks = dbt;
    plan.warp_tasks = dwt;
    CHECK_CUDA(cudaMalloc((void**)&doff, sizeof(int64_t) * (S + 1)));
    CHECK_CUDA(cudaMalloc((void**)&ddeg, sizeof(int32_t) * S));
    CHECK_CUDA(cudaMemcpy(doff, hoff, sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(ddeg, hdeg, sizeof(int32_t) * S, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMalloc((void**)&dBX, sizeof(double) * S * (m_max + 1)));
    CHECK_CUDA(cudaMalloc((void**)&dbst, sizeof(int32_t) * S));
    size_t bws_bytes = lsefit_batched_workspace_size(&plan);
    void* bws;
    CHECK_CUDA(cudaMalloc(&bws, bws_bytes));
    lsefit_batch batch;
    memset(&batch, 0, sizeof(batch));
    batch.x = dx;
    batch.y = dy;
    batch.offsets = doff;
    batch.degree = ddeg;
    batch.interval = NULL;
    batch.num_series = S;
    batch.m_max = m_max;
    batch.dtype = LSEFIT_F32;
    batch.accum = LSEFIT_ACCUM_COMP;
    CHECK_LSE(lsefit_fit_batched(&batch, &plan, dBX, NULL, NULL, NULL, dbst, bws, bws_bytes, NULL));
    double* hBX = (double*)malloc(sizeof(double) * S * (m_max + 1));
    int32_t* hbst = (int32_t*)malloc(sizeof(int32_t) * S);
    CHECK_CUDA(cudaMemcpy(hBX, dBX, sizeof(double) * S * (m_max + 1), cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(hbst, dbst, sizeof(int32_t) * S, cudaMemcpyDeviceToHost));
    for (long s = 0; s < S; ++s) {
        printf("batch %ld %d", s, hbst[s]);
        for (int j = 0; j <= hdeg[s]; ++j) printf(" %.17g", hBX[s * (m_max + 1) + j]);
        printf("\n");
    }
    return 0;
}
