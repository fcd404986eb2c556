// qs3_hphi_common.cuh -- device helpers shared by the H Phi kernels
// (qs3_hphi.cu) and the stored-term H Phi (qs3_terms.cu): vector-type traits,
// fused multiply-adds, the shared-memory layout of the row kernels, the
// diagonal constants and coupling tables in the vector's precision.
#pragma once

#include <algorithm>
#include <atomic>

#include "qs3_internal.cuh"

namespace qs3 {

template <typename VT> struct VTr;
template <> struct VTr<float> { using R = float; using C = float2; static constexpr bool cplx = false; };
template <> struct VTr<double> { using R = double; using C = double2; static constexpr bool cplx = false; };
template <> struct VTr<float2> { using R = float; using C = float2; static constexpr bool cplx = true; };
template <> struct VTr<double2> { using R = double; using C = double2; static constexpr bool cplx = true; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// acc += coef * x: complex coefficient (explicit fma chains: four fused
// multiply-adds per complex product instead of multiply, fma and add per part)
__device__ __forceinline__ void acc_add(float2 &acc, float2 coef, float2 x) {
    acc.x = fmaf(coef.x, x.x, acc.x);
    acc.x = fmaf(-coef.y, x.y, acc.x);
    acc.y = fmaf(coef.x, x.y, acc.y);
    acc.y = fmaf(coef.y, x.x, acc.y);
}
__device__ __forceinline__ void acc_add(double2 &acc, double2 coef, double2 x) {
    acc.x = fma(coef.x, x.x, acc.x);
    acc.x = fma(-coef.y, x.y, acc.x);
    acc.y = fma(coef.x, x.y, acc.y);
    acc.y = fma(coef.y, x.x, acc.y);
}
// acc += c * x with a real coefficient; a real x touches acc.x only
__device__ __forceinline__ void madd_r(float2 &acc, float c, float x) { acc.x = fmaf(c, x, acc.x); }
__device__ __forceinline__ void madd_r(double2 &acc, double c, double x) { acc.x = fma(c, x, acc.x); }
__device__ __forceinline__ void madd_r(float2 &acc, float c, float2 x) {
    acc.x = fmaf(c, x.x, acc.x);
    acc.y = fmaf(c, x.y, acc.y);
}
__device__ __forceinline__ void madd_r(double2 &acc, double c, double2 x) {
    acc.x = fma(c, x.x, acc.x);
    acc.y = fma(c, x.y, acc.y);
}
__device__ __forceinline__ void store(float *p, float2 v) { *p = v.x; }
__device__ __forceinline__ void store(double *p, double2 v) { *p = v.x; }
__device__ __forceinline__ void store(float2 *p, float2 v) { *p = v; }
__device__ __forceinline__ void store(double2 *p, double2 v) { *p = v; }

template <typename VT> __device__ __forceinline__ const typename VTr<VT>::R *jxy_table(const LatView &L);
template <> __device__ __forceinline__ const float *jxy_table<float>(const LatView &L) { return L.adj_jxy_f; }
template <> __device__ __forceinline__ const float *jxy_table<float2>(const LatView &L) { return L.adj_jxy_f; }
template <> __device__ __forceinline__ const double *jxy_table<double>(const LatView &L) { return L.adj_jxy; }
template <> __device__ __forceinline__ const double *jxy_table<double2>(const LatView &L) { return L.adj_jxy; }

struct SmemLayout {
    uint64_t *sC;
    uint32_t *sxyz;
    void *snorm;    // sqrt table: [0..8] sqrt(s), [9..17] 1/sqrt(s)
    void *sph;      // k-sectors: the current sector's per-site phases (vector precision)
};

// layout (must match row_kernel_smem): binomial rows 0..nd+2 | coordinates
// (k only) | sqrt table | per-site phases (k only)
__device__ __forceinline__ SmemLayout carve(const LatView &L, unsigned char *smem) {
    SmemLayout s;
    s.sC = (uint64_t *)smem;
    s.sxyz = (uint32_t *)(s.sC + (L.nd + 3) * L.np1);
    size_t off = (size_t)(L.nd + 3) * L.np1 * 8 + (L.has_k ? (size_t)L.N * 4 : 0);
    off = (off + 15) & ~(size_t)15;
    s.snorm = smem + off;
    off += 18 * sizeof(double);
    off = (off + 15) & ~(size_t)15;
    s.sph = smem + off;
    return s;
}

template <typename R> __device__ __forceinline__ R diag_c0(const LatView &L);
template <> __device__ __forceinline__ double diag_c0<double>(const LatView &L) { return L.c0; }
template <> __device__ __forceinline__ float diag_c0<float>(const LatView &L) { return L.c0f; }
template <typename R> __device__ __forceinline__ R diag_u(const LatView &L, int i);
template <> __device__ __forceinline__ double diag_u<double>(const LatView &L, int i) { return __ldg(L.u + i); }
template <> __device__ __forceinline__ float diag_u<float>(const LatView &L, int i) { return __ldg(L.u_f + i); }
template <typename R> __device__ __forceinline__ R diag_jz(const LatView &L, int q);
template <> __device__ __forceinline__ double diag_jz<double>(const LatView &L, int q) { return __ldg(L.adj_jz + q); }
template <> __device__ __forceinline__ float diag_jz<float>(const LatView &L, int q) { return __ldg(L.adj_jz_f + q); }

template <typename CT> __device__ __forceinline__ const CT *phase_table(const SecView &sv);
template <> __device__ __forceinline__ const double2 *phase_table<double2>(const SecView &sv) { return sv.ph64; }
template <> __device__ __forceinline__ const float2 *phase_table<float2>(const SecView &sv) { return sv.ph32; }

// ------------------------------------------------ host: launch shape

// SM count of the current device (the one the basis lives on)
static inline int num_sms() {
    static std::atomic<int> nsm{0};
    int n = nsm.load(std::memory_order_relaxed);
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        nsm.store(n, std::memory_order_relaxed);
    }
    return n;
}

// persistent grid: resident blocks per SM x SMs, capped by the tile count.
// cache packs (smem + 1) << 32 | blocks per SM, so concurrent callers read a
// consistent pair; the shared-memory attribute is always MAX_DYN_SMEM.
template <typename KF>
static int launch_rows(KF kern, Basis &B, size_t smem, std::atomic<unsigned long long> &cache, int *grid_out,
                       int *occ_out = nullptr) {
    const unsigned long long c = cache.load(std::memory_order_acquire);
    int nb;
    if ((c >> 32) != (unsigned long long)smem + 1) {
        QS3_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        QS3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NTHREADS, smem));
        nb = std::max(nb, 1);
        cache.store(((unsigned long long)smem + 1) << 32 | (unsigned)nb, std::memory_order_release);
    } else {
        nb = (int)(c & 0xffffffffu);
    }
    int grid = std::min(B.ntiles, nb * num_sms());
    *grid_out = std::max(grid, 1);
    if (occ_out) *occ_out = nb;
    return QS3_OK;
}

// autotuner for the persistent grid: on the first direct launch for a basis
// and vector type, time the kernel with 1..4 fewer resident blocks per SM
// than the occupancy limit (rows in flight per SM) and keep the fastest.
// H Phi is a pure function of phi, so the trial launches only rewrite psi.
// launch(grid) enqueues one launch on st.
template <typename LF>
static int tune_blocks(Basis &B, int occ, cudaStream_t st, int &best_bps, LF launch) {
    const int nsm = num_sms();
    best_bps = occ;
    if (B.ntiles < 2 * nsm || occ <= 1) return QS3_OK;
    cudaEvent_t e0, e1;
    QS3_CUDA(cudaEventCreate(&e0));
    QS3_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int rc = QS3_OK;
    for (int b = occ; b >= std::max(1, occ - 3) && rc == QS3_OK; --b) {
        const int grid = std::min(B.ntiles, b * nsm);
        float tmin = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            launch(grid);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) { rc = QS3_ERR_CUDA; break; }
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = QS3_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 || b < occ) tmin = std::min(tmin, ms);   // the very first launch warms up
        }
        if (tmin < best) { best = tmin; best_bps = b; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != QS3_OK) return set_err(rc, "H Phi autotuning launch failed");
    return QS3_OK;
}

}  // namespace qs3
