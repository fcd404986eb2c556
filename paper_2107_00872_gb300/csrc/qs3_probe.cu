// qs3_probe.cu -- throughput microbenchmarks of this GPU's arithmetic pipes
// (fp64 FMA, fp32 FMA, integer multiply-add, integer logic/add) and its warp
// instruction issue rate, the denominators of the ALU rooflines that the
// benchmark reports.  The paper has no counterpart (its code runs on CPUs).
//
// Each probe launches 8 blocks of 256 threads per SM (full occupancy); every
// thread runs 8 independent dependency chains of one instruction kind, so
// latency is hidden and the pipe under test is the only limit.  Timing uses
// CUDA events on the caller's stream around the second of two launches.
// Results only feed measurement; nothing in the solver depends on them.
#include <cuda_runtime.h>

#include <cstring>

#include "qs3_internal.cuh"

namespace qs3 {

constexpr int PROBE_CHAINS = 8;

// KIND 0: fp64 fma, 1: fp32 fma, 2: int32 multiply-add, 3: int32 xor + add
template <int KIND>
__global__ void __launch_bounds__(256) k_probe(int iters, double md, double cd, unsigned mi, unsigned ci,
                                               double *__restrict__ sink) {
    double acc = 0.0;
    if constexpr (KIND == 0) {
        double a[PROBE_CHAINS];
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (double)(threadIdx.x + k);
#pragma unroll 1
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], md, cd);
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) acc += a[k];
    } else if constexpr (KIND == 1) {
        float a[PROBE_CHAINS];
        const float mf = (float)md, cf = (float)cd;
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
#pragma unroll 4
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], mf, cf);
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) acc += a[k];
    } else {
        unsigned a[PROBE_CHAINS];
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = threadIdx.x * 2654435761u + k;
#pragma unroll 4
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) {
                // non-linear recurrences (a linear one would be folded across
                // iterations by the compiler): one multiply-add, or xor + add
                if constexpr (KIND == 2) a[k] = a[k] * a[k] + ci;
                else a[k] = (a[k] ^ ci) + a[k];
            }
        unsigned s = 0;
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) s ^= a[k];
        // a runtime comparison: a test the compiler could decide (a converted
        // integer is never -1.0) would let it drop the chains
        if (s == mi) sink[blockIdx.x] = (double)s;
        return;
    }
    // the store depends on every chain, so nothing is optimised away
    if (acc == -1.0) sink[blockIdx.x] = acc;
}

template <int KIND>
static int probe_one(int iters, int blocks, cudaStream_t st, double *sink, double &ops_per_s) {
    cudaEvent_t e0, e1;
    QS3_CUDA(cudaEventCreate(&e0));
    QS3_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    int rc = QS3_OK;
    for (int rep = 0; rep < 2 && rc == QS3_OK; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = QS3_ERR_CUDA; break; }
        k_probe<KIND><<<blocks, 256, 0, st>>>(iters, 0.999999999, 1e-9, 1664525u, 1013904223u, sink);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) { rc = QS3_ERR_CUDA; break; }
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = QS3_ERR_CUDA;
            break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != QS3_OK) return set_err(rc, "probe kernel %d failed", KIND);
    const double per_iter = (KIND == 3 ? 2.0 : 1.0) * PROBE_CHAINS;
    ops_per_s = (double)blocks * 256.0 * iters * per_iter / (1e-3 * ms);
    return QS3_OK;
}

}  // namespace qs3

using namespace qs3;

extern "C" int qs3_probe_peaks(qs3_peaks *out, void *stream) {
    clear_err();
    if (!out) return set_err(QS3_ERR_INVALID_ARG, "NULL output");
    memset(out, 0, sizeof(*out));
    int dev = 0, sms = 0;
    QS3_CUDA(cudaGetDevice(&dev));
    QS3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = sms * 8;
    DevBuf sink;
    QS3_TRY(sink.alloc((size_t)blocks * sizeof(double)));
    double *s = sink.as<double>();
    // iteration counts sized for ~10-30 ms per launch at the nominal rates
    QS3_TRY(probe_one<0>(2048, blocks, st, s, out->fp64_fma_per_s));
    QS3_TRY(probe_one<1>(131072, blocks, st, s, out->fp32_fma_per_s));
    QS3_TRY(probe_one<2>(32768, blocks, st, s, out->int_mad_per_s));
    QS3_TRY(probe_one<3>(32768, blocks, st, s, out->int_alu_per_s));
    // one warp instruction per 32 lanes: the fp32 FMA probe issues nothing else
    out->issue_per_s = out->fp32_fma_per_s / 32.0;
    out->n_sms = sms;
    return QS3_OK;
}
