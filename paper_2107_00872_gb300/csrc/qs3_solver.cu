// qs3_solver.cu -- conventional Lanczos and thick-restart Lanczos (Alg. 10),
// batched over the sectors of a basis.
//
// All sectors advance in lock step on one concatenated vector: every kernel
// covers all sectors in one launch, reductions are per sector (fixed-order
// two-stage trees, so results are deterministic), and a per-sector active
// flag removes converged sectors from every launch.  The Lanczos vectors
// Psi live in one device array (vector j at offset j * total_dim).
//
// One Lanczos step (Alg. 10 lines 5-11) for x: v = H psi_x; the three-term
// part removes the components along psi_{x-1}, psi_x (coefficients by dot
// product, alpha_x among them), then one classical Gram-Schmidt pass against
// psi_0..psi_x removes the O(eps) rest (two full passes on the first step
// after a thick restart); beta_x = |v|; psi_{x+1} = v / beta_x.  Dot
// products, norms and the Gram-Schmidt coefficients are fp64-accurate
// (binary64 or double-float sums) even when the vectors are fp32.
//
// Engines: the binary64 engine (qs3_engine64.cuh, precision QS3_F64), the
// double-float engine (Engine with dfh, precision QS3_C128DF on k-sector
// bases) and the fp32 engine (Engine<float / float2>, the fp32 phase of
// precision QS3_F32).  The convergence checks of conventional Lanczos (the
// tridiagonal T) run on the device (Sturm multisection + inverse
// iteration), so the whole loop can replay as one CUDA graph; the arrowhead
// T of the thick restart is diagonalised on the host (cyclic Jacobi).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "qs3_internal.cuh"
#include "qs3_df.cuh"

namespace qs3 {

// ------------------------------------------------------------ element access
__device__ __forceinline__ double2 ld2(const float *p) { return make_double2((double)*p, 0.0); }
__device__ __forceinline__ double2 ld2(const double *p) { return make_double2(*p, 0.0); }
__device__ __forceinline__ double2 ld2(const float2 *p) { float2 v = *p; return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 ld2(const double2 *p) { return *p; }
__device__ __forceinline__ void st2(float *p, double2 v) { *p = (float)v.x; }
__device__ __forceinline__ void st2(double *p, double2 v) { *p = v.x; }
__device__ __forceinline__ void st2(float2 *p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void st2(double2 *p, double2 v) { *p = v; }
// conj(a) * b
__device__ __forceinline__ double2 cdot(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cmad(double2 acc, double2 a, double2 b) {   // acc + a * b
    return make_double2(acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x);
}

template <typename VT> struct Is64 { static constexpr bool v = false; };
template <> struct Is64<double> { static constexpr bool v = true; };
template <> struct Is64<double2> { static constexpr bool v = true; };
template <typename VT> struct IsC { static constexpr bool v = false; };
template <> struct IsC<float2> { static constexpr bool v = true; };
template <> struct IsC<double2> { static constexpr bool v = true; };
template <typename VT> struct Wide { using T = double; };
template <> struct Wide<float2> { using T = double2; };
template <> struct Wide<double2> { using T = double2; };

struct ChunkInfo {
    int s;
    uint64_t base;   // first row of the chunk in the concatenated vector
    int n;           // rows in the chunk
};

__device__ __forceinline__ ChunkInfo chunk_info(const SecView *secs, const int *chunk0, int S, int c) {
    ChunkInfo ci;
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (chunk0[mid] <= c) lo = mid; else hi = mid - 1;
    }
    ci.s = lo;
    const uint64_t r0 = (uint64_t)(c - chunk0[lo]) * BROWS;
    ci.base = secs[lo].off + r0;
    const uint64_t rem = secs[lo].dim - r0;
    ci.n = (int)(rem < (uint64_t)BROWS ? rem : (uint64_t)BROWS);
    return ci;
}

// graph mode: the step index lives in device memory
__global__ void k_setx(int *dx, int x) { *dx = x; }
__global__ void k_advance(int *dx) { *dx += 1; }

constexpr int RPT = BROWS / NTHREADS;   // rows per thread
constexpr int JB = 32;                  // dot products per reduction batch

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// part[c * m + j] = sum over the chunk's rows of conj(V_{j0+j}) w; vector j
// starts at V + j * ld (ld may be negative)
template <typename VT>
__global__ void __launch_bounds__(NTHREADS) k_mdot(const VT *__restrict__ V, int64_t ld, int j0, int m,
                                                   const VT *__restrict__ w, const SecView *__restrict__ secs,
                                                   const int *__restrict__ chunk0, int S,
                                                   const int *__restrict__ active, double2 *__restrict__ part,
                                                   const int *__restrict__ dx = nullptr) {
    __shared__ double2 red[NTHREADS / 32][JB];
    if (dx) {                         // graph mode: psi_{x-1}, psi_x, or psi_0 alone at x = 0
        if (*dx == 0) { V += ld; m = 1; } else { m = 2; }
    }
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    double2 wv[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        wv[k] = (r < ci.n) ? ld2(w + ci.base + r) : make_double2(0.0, 0.0);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int jb = 0; jb < m; jb += JB) {
        const int nj = min(JB, m - jb);
        for (int jj = 0; jj < nj; ++jj) {
            const VT *vj = V + (int64_t)(j0 + jb + jj) * ld + ci.base;
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = threadIdx.x + k * NTHREADS;
                if (r < ci.n) {
                    const double2 a = ld2(vj + r), d = cdot(a, wv[k]);
                    acc.x += d.x;
                    acc.y += d.y;
                }
            }
            acc = warp_sum2(acc);
            if (lane == 0) red[warp][jj] = acc;
        }
        __syncthreads();
        if (threadIdx.x < nj) {
            double2 t = make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < NTHREADS / 32; ++q) { t.x += red[q][threadIdx.x].x; t.y += red[q][threadIdx.x].y; }
            part[(uint64_t)blockIdx.x * m + jb + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[s * ldo + j] = sum of part[c * m + j] over the chunks of sector s (one block per (j, s))
// out[s * ldo + j] = sum of part[c * m + j] over the chunks of sector s; block
// (x, s) takes j = x, x + gridDim.x, ...  Graph mode (dx): ring = the
// three-term pass (m = 1 at x = 0, else 2, out at x - 1), otherwise the full
// pass (m = x + 1)
__global__ void k_reduce(const double2 *__restrict__ part, int m, const int *__restrict__ chunk0,
                         const int *__restrict__ active, double2 *__restrict__ out, int ldo,
                         const int *__restrict__ dx = nullptr, bool ring = false) {
    const int s = blockIdx.y;
    if (dx) {
        const int x = *dx;
        m = ring ? (x > 0 ? 2 : 1) : x + 1;
        if (ring) out += max(0, x - 1);
    }
    if (active && !active[s]) return;
    __shared__ double2 red[NTHREADS / 32];
    for (int j = blockIdx.x; j < m; j += gridDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int c = chunk0[s] + threadIdx.x; c < chunk0[s + 1]; c += blockDim.x) {
            double2 v = part[(uint64_t)c * m + j];
            acc.x += v.x;
            acc.y += v.y;
        }
        acc = warp_sum2(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double2 t = make_double2(0.0, 0.0);
            for (int q = 0; q < NTHREADS / 32; ++q) { t.x += red[q].x; t.y += red[q].y; }
            out[(uint64_t)s * ldo + j] = t;
        }
        __syncthreads();
    }
}

// w -= sum_j V_{j0+j} coef[s][j]; optionally part[c] = sum |w|^2 over the chunk
template <typename VT>
__global__ void __launch_bounds__(NTHREADS) k_mupdate(VT *__restrict__ w, const VT *__restrict__ V, int64_t ld,
                                                      int j0, int m, const double2 *__restrict__ coef, int ldc,
                                                      const SecView *__restrict__ secs,
                                                      const int *__restrict__ chunk0, int S,
                                                      const int *__restrict__ active, double2 *__restrict__ part,
                                                      const int *__restrict__ dx = nullptr) {
    extern __shared__ double2 sco[];
    __shared__ double red[NTHREADS / 32];
    if (dx) {                         // graph mode: psi_{x-1}, psi_x, or psi_0 alone at x = 0
        if (*dx == 0) { V += ld; m = 1; } else { m = 2; }
        coef += max(0, *dx - 1);
    }
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    for (int j = threadIdx.x; j < m; j += blockDim.x) sco[j] = coef[(uint64_t)ci.s * ldc + j];
    __syncthreads();
    double nrm = 0.0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            double2 acc = ld2(w + ci.base + r);
            const VT *vp = V + (int64_t)j0 * ld + ci.base + r;
            for (int j = 0; j < m; ++j) {
                const double2 a = ld2(vp + (int64_t)j * ld), c = sco[j];
                acc.x -= a.x * c.x - a.y * c.y;
                acc.y -= a.x * c.y + a.y * c.x;
            }
            st2(w + ci.base + r, acc);
            const double2 q = ld2(w + ci.base + r);   // norm of the stored (rounded) value
            nrm += q.x * q.x + q.y * q.y;
        }
    }
    if (part) {
#pragma unroll
        for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < NTHREADS / 32; ++q) t += red[q];
            part[blockIdx.x] = make_double2(t, 0.0);
        }
    }
}

// per-sector scalars after a step: alpha_x, beta_x (with breakdown), 1/beta
__global__ void k_step_scalars(int S, int x, int cap, const double2 *__restrict__ h, const double2 *__restrict__ nrm2,
                               const int *__restrict__ active, double *__restrict__ alpha, double *__restrict__ beta,
                               double *__restrict__ inv, double brk, const int *__restrict__ dx = nullptr) {
    if (dx) x = *dx;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || (active && !active[s])) return;
    const double a = h[(uint64_t)s * cap + x].x;
    double b = sqrt(fmax(nrm2[s].x, 0.0));
    const double bprev = x > 0 ? beta[(uint64_t)s * cap + x - 1] : 0.0;
    if (!(b > brk * (fabs(a) + bprev)) || !isfinite(b)) b = 0.0;      // invariant subspace reached
    alpha[(uint64_t)s * cap + x] = a;
    beta[(uint64_t)s * cap + x] = b;
    inv[s] = b > 0.0 ? 1.0 / b : 0.0;
}

// ---------------------------------------------- fp32 vectors, fp64-accurate
// For fp32 / complex64 vectors the dot products and the Gram-Schmidt updates
// are carried on the fp32 units in double-float form (a value is hi + lo,
// two floats): products of two floats are exact as p + e with e =
// fma(a, b, -p), sums use the error-free two-sum.  This keeps ~48 bits, i.e.
// fp64-class accumulation, at fp32 throughput (GB300 executes fp64 at a
// small fraction of its fp32 rate).  Partial sums leave each thread in fp64.

template <typename VT> struct F32c { static constexpr bool v = false; };
template <> struct F32c<float2> { static constexpr bool v = true; };

__device__ __forceinline__ float2 ldf(const float *p) { return make_float2(*p, 0.f); }
__device__ __forceinline__ float2 ldf(const float2 *p) { return *p; }

// w -= sum_j V_{j0+j} coef[s][j] in double-float, rounded once to fp32;
// optionally part[c] = sum |w|^2 over the chunk
template <typename VT>
__global__ void __launch_bounds__(NTHREADS) k_mupdate32(VT *__restrict__ w, const VT *__restrict__ V, uint64_t D,
                                                        int j0, int m, const double2 *__restrict__ coef, int ldc,
                                                        const SecView *__restrict__ secs,
                                                        const int *__restrict__ chunk0, int S,
                                                        const int *__restrict__ active, double2 *__restrict__ part) {
    extern __shared__ float4 scf[];   // per j: (re.hi, re.lo, im.hi, im.lo)
    __shared__ double red[NTHREADS / 32];
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double2 c = coef[(uint64_t)ci.s * ldc + j];
        const float rh = (float)c.x, ih = (float)c.y;
        scf[j] = make_float4(rh, (float)(c.x - (double)rh), ih, (float)(c.y - (double)ih));
    }
    __syncthreads();
    dfl nr = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            const float2 w0 = ldf(w + ci.base + r);
            dfl re = {w0.x, 0.f}, im = {w0.y, 0.f};
            const VT *vp = V + (uint64_t)j0 * D + ci.base + r;
            for (int j = 0; j < m; ++j) {
                const float2 a = ldf(vp + (uint64_t)j * D);
                const float4 c = scf[j];
                // w -= a * c: re -= a.x c.x - a.y c.y ; im -= a.x c.y + a.y c.x
                re = df_fma2(re, -a.x, c.x, c.y);
                if (F32c<VT>::v) {
                    re = df_fma2(re, a.y, c.z, c.w);
                    im = df_fma2(im, -a.x, c.z, c.w);
                    im = df_fma2(im, -a.y, c.x, c.y);
                }
            }
            const float2 out = make_float2(re.hi + re.lo, im.hi + im.lo);
            if (F32c<VT>::v) ((float2 *)w)[ci.base + r] = out;
            else ((float *)w)[ci.base + r] = out.x;
            nr = df_fma(nr, out.x, out.x);
            nr = df_fma(nr, out.y, out.y);
        }
    }
    if (part) {
        double v = df_d(nr);
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < NTHREADS / 32; ++q) t += red[q];
            part[blockIdx.x] = make_double2(t, 0.0);
        }
    }
}

// w *= inv[s] (per sector)
template <typename VT>
__global__ void __launch_bounds__(NTHREADS) k_scale(VT *__restrict__ w, const double *__restrict__ inv,
                                                    const SecView *__restrict__ secs, const int *__restrict__ chunk0,
                                                    int S, const int *__restrict__ active) {
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const double f = inv[ci.s];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            double2 v = ld2(w + ci.base + r);
            v.x *= f;
            v.y *= f;
            st2(w + ci.base + r, v);
        }
    }
}

// sum |w|^2 per chunk
template <typename VT>
__global__ void __launch_bounds__(NTHREADS) k_norm2(const VT *__restrict__ w, const SecView *__restrict__ secs,
                                                    const int *__restrict__ chunk0, int S,
                                                    const int *__restrict__ active, double2 *__restrict__ part) {
    __shared__ double red[NTHREADS / 32];
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    double nrm = 0.0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            const double2 q = ld2(w + ci.base + r);
            nrm += q.x * q.x + q.y * q.y;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < NTHREADS / 32; ++q) t += red[q];
        part[blockIdx.x] = make_double2(t, 0.0);
    }
}

__global__ void k_inv_sqrt(int S, const double2 *__restrict__ n2, double *__restrict__ inv) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) inv[s] = n2[s].x > 0.0 ? 1.0 / sqrt(n2[s].x) : 0.0;
}

// SplitMix64 output function (Steele, Lea, Flood 2014)
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Box-Muller normal from counters 2i, 2i+1 of the stream seeded by `seed`
__device__ __forceinline__ double gauss(uint64_t seed, uint64_t i) {
    const double u1 = ((double)(splitmix64(seed ^ (2 * i)) >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = ((double)(splitmix64(seed ^ (2 * i + 1)) >> 11) + 1.0) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// start vector of sector s: seed + s, element i (imaginary part from counters offset by dim)
template <typename VT>
__global__ void __launch_bounds__(NTHREADS) k_random(VT *__restrict__ w, uint64_t seed,
                                                     const SecView *__restrict__ secs,
                                                     const int *__restrict__ chunk0, int S) {
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    const uint64_t sseed = seed + (uint64_t)ci.s;
    const uint64_t r0 = ci.base - secs[ci.s].off;
    const uint64_t d = secs[ci.s].dim;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            const uint64_t i = r0 + r;
            double2 v = make_double2(gauss(sseed, i), 0.0);
            if (IsC<VT>::v) v.y = gauss(sseed, d + i);
            st2(w + ci.base + r, v);
        }
    }
}

// dst = (VT) src for the rows of active sectors
template <typename VT, typename ST>
__global__ void __launch_bounds__(NTHREADS) k_convert(VT *__restrict__ dst, const ST *__restrict__ src,
                                                      const SecView *__restrict__ secs,
                                                      const int *__restrict__ chunk0, int S,
                                                      const int *__restrict__ active) {
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) st2(dst + ci.base + r, ld2(src + ci.base + r));
    }
}

// out_y[r] = sum_x V_x[r] C[s][x][y] (y < nout <= 16), rows of sectors with mask[s] != 0
constexpr int MAXOUT = 16;
template <typename VT, typename OT>
__global__ void __launch_bounds__(NTHREADS) k_combine(OT *__restrict__ out, uint64_t ldo, const VT *__restrict__ V,
                                                      uint64_t D, int nin, int nout, const double *__restrict__ C,
                                                      int ldc, const SecView *__restrict__ secs,
                                                      const int *__restrict__ chunk0, int S,
                                                      const int *__restrict__ mask) {
    extern __shared__ double sc[];
    __shared__ int nx;
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (mask && !mask[ci.s]) return;
    const double *Cs = C + (uint64_t)ci.s * ldc;
    if (threadIdx.x == 0) nx = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nin * nout; i += blockDim.x) {
        sc[i] = Cs[i];
        if (Cs[i] != 0.0) atomicMax(&nx, i / nout + 1);
    }
    __syncthreads();
    nin = nx;      // vectors past the sector's last nonzero coefficient may be unwritten
#pragma unroll 1
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r >= ci.n) continue;
        double2 acc[MAXOUT];
#pragma unroll
        for (int y = 0; y < MAXOUT; ++y) acc[y] = make_double2(0.0, 0.0);
        for (int x = 0; x < nin; ++x) {
            const double2 a = ld2(V + (uint64_t)x * D + ci.base + r);
#pragma unroll
            for (int y = 0; y < MAXOUT; ++y)
                if (y < nout) {
                    const double c = sc[x * nout + y];
                    acc[y].x += a.x * c;
                    acc[y].y += a.y * c;
                }
        }
#pragma unroll
        for (int y = 0; y < MAXOUT; ++y)
            if (y < nout) st2(out + (uint64_t)y * ldo + ci.base + r, acc[y]);
    }
}

// ------------------------------------ fp64 Lanczos vectors, double-float store
// The Krylov basis of an fp64 solve is stored as double-float pairs: an
// element v is kept as hi = fl32(v), lo = fl32(v - hi), 48 significant bits
// in the same 8 bytes.  The Gram-Schmidt pass over all kept vectors (the
// reorthogonalisation of Alg. 10) then runs on the fp32 units with
// error-free products (fma) and two-sums; the fp64 unit -- a small fraction
// of the fp32 rate on this GPU -- only sees one conversion per row and
// kernel.  Complex k-sector solves (the double-float engine, Engine::dfh)
// keep w = H psi_x in double-float as well and run H (k_hphi_df), the
// three-term part and the scaling on the fp32 units; real and U(1) solves
// apply H and the three-term part to exact fp64 copies of psi_{x-1}, psi_x.
// The 2^-48 rounding only bounds how far below fp64 epsilon the
// orthogonality of the basis can be pushed.
template <typename VT> struct DfS { using T = VT; };     // fp32 vectors: stored as they are
template <> struct DfS<double> { using T = float2; };    // (hi, lo)
template <> struct DfS<double2> { using T = float4; };   // (re.hi, re.lo, im.hi, im.lo)

// Layout of a stored vector (a slot of D elements).  Real: (hi, lo) pairs.
// Complex: two planes, the D hi pairs (re.hi, im.hi) then the D lo pairs
// (re.lo, im.lo), so a pass that needs only the hi words (the update with
// O(eps) coefficients) reads half the bytes.  Values are handed around as
// float4 (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ float4 ld_st(const float2 *slot, uint64_t, uint64_t r) {
    const float2 v = slot[r];
    return make_float4(v.x, v.y, 0.f, 0.f);
}
__device__ __forceinline__ float4 ld_st(const float4 *slot, uint64_t D, uint64_t r) {
    const float2 *h = (const float2 *)slot;
    const float2 a = h[r], b = h[D + r];
    return make_float4(a.x, b.x, a.y, b.y);
}
// the hi words only: (re.hi, im.hi)
__device__ __forceinline__ float2 ld_st_hi(const float2 *slot, uint64_t, uint64_t r) { return make_float2(slot[r].x, 0.f); }
__device__ __forceinline__ float2 ld_st_hi(const float4 *slot, uint64_t, uint64_t r) { return ((const float2 *)slot)[r]; }
__device__ __forceinline__ void st_st(float2 *slot, uint64_t, uint64_t r, float4 v) { slot[r] = make_float2(v.x, v.y); }
__device__ __forceinline__ void st_st(float4 *slot, uint64_t D, uint64_t r, float4 v) {
    float2 *h = (float2 *)slot;
    h[r] = make_float2(v.x, v.z);
    h[D + r] = make_float2(v.y, v.w);
}
// the working vector w of a Gram-Schmidt pass: fp64 (split on load) or
// already double-float (the double-float engine of complex k-sector solves)
__device__ __forceinline__ float4 ld_w(const double *p) { return split2(ld2(p)); }
__device__ __forceinline__ float4 ld_w(const double2 *p) { return split2(ld2(p)); }
__device__ __forceinline__ float4 ld_w(const float4 *p) { return *p; }
// fp32 vectors (the fp32 engine) are double-float values with lo = 0
__device__ __forceinline__ float4 ld_w(const float *p) { return make_float4(*p, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 ld_w(const float2 *p) { const float2 v = *p; return make_float4(v.x, 0.f, v.y, 0.f); }
// graph mode (dx): the three-term pass takes vectors x - 1, x (m = 2, x >= 1),
// the full pass vectors 0 .. x
// the stored vectors a kernel of the captured step reads, from x = *dx:
// ring 0: psi_0 .. psi_x; ring 1: psi_{x-1}, psi_x; ring 2: psi_x alone
__device__ __forceinline__ void graph_range(const int *dx, int ring, int &j0, int &m) {
    if (!dx) return;
    if (ring == 2) { j0 = *dx; m = 1; }
    else if (ring) { j0 = *dx - 1; m = 2; }
    else { j0 = 0; m = *dx + 1; }
}


// part[c * m + j] = conj(V_{j0+j}) . w over the chunk as double-float
// (re.hi, re.lo, im.hi, im.lo); V double-float, w fp64.  Vectors go in groups
// of 8: every thread leaves its partial sums in shared memory, then warp q
// reduces vector q of the group (one shuffle tree per vector and block
// instead of one per vector and warp).  NV vectors per pass have all their
// loads in flight together (the staging depth, chosen by the autotuner).
constexpr int GDF = NTHREADS / 32;
template <typename VT, int NV, typename WV = VT>
__global__ void __launch_bounds__(NTHREADS, NV == 1 ? 4 : NV == 2 ? 2 : 1) k_mdot_df(const typename DfS<VT>::T *__restrict__ V, uint64_t D, int j0,
                                                      int m, const WV *__restrict__ w,
                                                      const SecView *__restrict__ secs,
                                                      const int *__restrict__ chunk0, int S,
                                                      const int *__restrict__ active, float4 *__restrict__ part,
                                                      const int *__restrict__ dx = nullptr, int ring = 0) {
    using ST = typename DfS<VT>::T;
    static_assert(GDF % NV == 0, "vectors per pass must divide the group");
    __shared__ float4 red[GDF][NTHREADS];
    graph_range(dx, ring, j0, m);
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    // w's rows stay in registers (NV > 1) or are re-read through L1 for each
    // vector (NV = 1: fewer registers, more resident blocks)
    float4 wv[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        wv[k] = (NV > 1 && r < ci.n) ? ld_w(w + ci.base + r) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a thread's rows are threadIdx.x + k NTHREADS: one base pointer per
    // vector and constant offsets (rows past the chunk end load zero)
    const int nk = (ci.n - (int)threadIdx.x + NTHREADS - 1) / NTHREADS;     // rows of this thread
    for (int jb = 0; jb < m; jb += GDF) {
        const int nj = min(GDF, m - jb);
        for (int jj = 0; jj < nj; jj += NV) {
            const ST *vb = V + (uint64_t)(j0 + jb + jj) * D;
            float4 a[NV][RPT];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const ST *vv = (jj + v < nj) ? vb + (uint64_t)v * D : vb;   // past the group: a repeat, discarded
                const uint64_t r0 = ci.base + threadIdx.x;
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    a[v][k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k < nk) {
                        if constexpr (Is64<VT>::v) a[v][k] = ld_st(vv, D, r0 + k * NTHREADS);
                        else a[v][k] = ld_w(vv + r0 + k * NTHREADS);      // fp32 store: lo = 0
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                dfl re = {0.f, 0.f}, im = {0.f, 0.f};
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    float4 b = wv[k];
                    if constexpr (NV == 1)
                        if (k < nk) b = ld_w(w + ci.base + threadIdx.x + k * NTHREADS);
                    const float4 x = a[v][k];
                    // conj(a) b = (a.r b.r + a.i b.i) + i (a.r b.i - a.i b.r)
                    df_mac(re, x.x, x.y, b.x, b.y);
                    if (IsC<VT>::v) {
                        df_mac(re, x.z, x.w, b.z, b.w);
                        df_mac(im, x.x, x.y, b.z, b.w);
                        df_mac(im, -x.z, -x.w, b.x, b.y);
                    }
                }
                if (jj + v < nj) {
                    re = df_norm(re);
                    im = df_norm(im);
                    red[jj + v][threadIdx.x] = make_float4(re.hi, re.lo, im.hi, im.lo);
                }
            }
        }
        __syncthreads();
        if (warp < nj) {
            dfl tr = {0.f, 0.f}, ti = {0.f, 0.f};
#pragma unroll
            for (int q = 0; q < NTHREADS / 32; ++q) {
                const float4 v = red[warp][lane + 32 * q];
                tr = df_sum(tr, {v.x, v.y});
                ti = df_sum(ti, {v.z, v.w});
            }
            tr = warp_sum_df(tr);
            if (IsC<VT>::v) ti = warp_sum_df(ti);
            if (lane == 0) part[(uint64_t)blockIdx.x * m + jb + warp] = make_float4(tr.hi, tr.lo, ti.hi, ti.lo);
        }
        __syncthreads();
    }
}

// k_reduce for double-float chunk partials (graph mode: the range of graph_range,
// written from out + j0)
__global__ void k_reduce_df(const float4 *__restrict__ part, int m, const int *__restrict__ chunk0,
                            const int *__restrict__ active, double2 *__restrict__ out, int ldo,
                            const int *__restrict__ dx = nullptr, int ring = 0) {
    const int s = blockIdx.y;
    if (dx) {
        int j0 = 0;
        graph_range(dx, ring, j0, m);
        out += j0;
    }
    if (active && !active[s]) return;
    // one warp per coefficient j: its lanes stride over the sector's chunks
    const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < m; j += gridDim.x * wpb) {
        double2 acc = make_double2(0.0, 0.0);
        for (int c = chunk0[s] + lane; c < chunk0[s + 1]; c += 32) {
            const float4 v = part[(uint64_t)c * m + j];
            acc.x += (double)v.x + (double)v.y;
            acc.y += (double)v.z + (double)v.w;
        }
        acc = warp_sum2(acc);
        if (lane == 0) out[(uint64_t)s * ldo + j] = acc;
    }
}

// w -= sum_j V_{j0+j} coef[s][j], subtracted from the fp64 w; optionally
// part[c] = sum |w|^2.  The sum u is formed in double-float over the stored
// basis; when the sector's coefficients are all below 2^-40 |w| (wn2 = |w|^2
// before this update; the second Gram-Schmidt pass, whose coefficients are
// O(eps |w|)), u is formed in plain fp32 from the hi words instead: its
// error, 2^-24 |u| <= 2^-24 * 2^-40 * sqrt(m) |w|, is below fp64 rounding of w.
// WV = float4: w itself is double-float (the double-float engine); the
// update and |w|^2 then stay on the fp32 units as well.
template <typename VT, typename WV = VT>
__global__ void __launch_bounds__(NTHREADS) k_mupdate_df(WV *__restrict__ w, const typename DfS<VT>::T *__restrict__ V,
                                                         uint64_t D, int j0, int m, const double2 *__restrict__ coef,
                                                         int ldc, const SecView *__restrict__ secs,
                                                         const int *__restrict__ chunk0, int S,
                                                         const int *__restrict__ active,
                                                         const double2 *__restrict__ wn2, double2 *__restrict__ part,
                                                         const int *__restrict__ dx = nullptr, int ring = 0) {
    using ST = typename DfS<VT>::T;
    constexpr bool WD = std::is_same<WV, float4>::value;
    if (dx) {
        graph_range(dx, ring, j0, m);
        if (ring) coef += j0;
    }
    extern __shared__ float4 scf[];   // per j: split coefficient (re.hi, re.lo, im.hi, im.lo)
    __shared__ double red[NTHREADS / 32];
    __shared__ unsigned cbits;
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    if (threadIdx.x == 0) cbits = 0u;
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double2 c = coef[(uint64_t)ci.s * ldc + j];
        scf[j] = split2(c);
        atomicMax(&cbits, __float_as_uint((float)(c.x * c.x + c.y * c.y)));   // non-negative: bits order as values
    }
    __syncthreads();
    const bool lite = wn2 && (double)__uint_as_float(cbits) <= 0x1p-80 * wn2[ci.s].x;
    dfl ur[RPT], ui[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) ur[k] = ui[k] = {0.f, 0.f};
    if (lite) {
        float2 uf[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) uf[k] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int j = 0; j < m; ++j) {
            const float4 c = scf[j];
            const ST *vj = V + (uint64_t)(j0 + j) * D;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = threadIdx.x + k * NTHREADS;
                if (r < ci.n) {
                    const float2 a = ld_st_hi(vj, D, ci.base + r);     // (re.hi, im.hi)
                    uf[k].x = fmaf(a.x, c.x, uf[k].x);
                    if (IsC<VT>::v) {
                        uf[k].x = fmaf(-a.y, c.z, uf[k].x);
                        uf[k].y = fmaf(a.x, c.z, uf[k].y);
                        uf[k].y = fmaf(a.y, c.x, uf[k].y);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            ur[k].hi = uf[k].x;
            ui[k].hi = uf[k].y;
        }
    } else {
#pragma unroll 2
        for (int j = 0; j < m; ++j) {
            const float4 c = scf[j];
            const ST *vj = V + (uint64_t)(j0 + j) * D;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = threadIdx.x + k * NTHREADS;
                if (r < ci.n) {
                    const float4 a = ld_st(vj, D, ci.base + r);
                    // u += a c: re += a.r c.r - a.i c.i ; im += a.r c.i + a.i c.r
                    df_mac(ur[k], a.x, a.y, c.x, c.y);
                    if (IsC<VT>::v) {
                        df_mac(ur[k], -a.z, -a.w, c.z, c.w);
                        df_mac(ui[k], a.x, a.y, c.z, c.w);
                        df_mac(ui[k], a.z, a.w, c.x, c.y);
                    }
                }
            }
        }
    }
    double nrm = 0.0;
    if constexpr (WD) {
        // w - u in double-float, |w|^2 accumulated per thread in double-float
        dfl n2 = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = threadIdx.x + k * NTHREADS;
            if (r < ci.n) {
                const float4 v = w[ci.base + r];
                const dfl re = df_sum({v.x, v.y}, {-ur[k].hi, -ur[k].lo});
                const dfl im = df_sum({v.z, v.w}, {-ui[k].hi, -ui[k].lo});
                w[ci.base + r] = make_float4(re.hi, re.lo, im.hi, im.lo);
                df_mac(n2, re.hi, re.lo, re.hi, re.lo);
                df_mac(n2, im.hi, im.lo, im.hi, im.lo);
            }
        }
        nrm = df_d(n2);
    } else {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = threadIdx.x + k * NTHREADS;
            if (r < ci.n) {
                double2 v = ld2(w + ci.base + r);
                v.x -= (double)ur[k].hi + (double)ur[k].lo;
                if (IsC<VT>::v) v.y -= (double)ui[k].hi + (double)ui[k].lo;
                st2(w + ci.base + r, v);
                nrm += v.x * v.x + v.y * v.y;
            }
        }
    }
    if (part) {
#pragma unroll
        for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < NTHREADS / 32; ++q) t += red[q];
            part[blockIdx.x] = make_double2(t, 0.0);
        }
    }
}

// w *= inv[s]; out = double-float copy of the scaled w
// (and, when hin is given, an interleaved double-float copy: the input of the
// double-float H Phi); D = the store's slot length
template <typename VT>
__global__ void __launch_bounds__(NTHREADS) k_scale_split(VT *__restrict__ w, typename DfS<VT>::T *__restrict__ out,
                                                          const double *__restrict__ inv,
                                                          const SecView *__restrict__ secs,
                                                          const int *__restrict__ chunk0, int S,
                                                          const int *__restrict__ active,
                                                          const int *__restrict__ dx, uint64_t D,
                                                          float4 *__restrict__ hin = nullptr) {
    if (dx) out += (uint64_t)(*dx + 1) * D;     // graph mode: out is the store's base, vector x + 1
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const double f = inv[ci.s];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            double2 v = ld2(w + ci.base + r);
            v.x *= f;
            v.y *= f;
            st2(w + ci.base + r, v);
            const float4 q = split2(v);
            st_st(out, D, ci.base + r, q);
            if (hin) hin[ci.base + r] = q;
        }
    }
}

// double-float engine, three-term update: w -= c_0 psi_{j0} + c_1 psi_{j0+1}
// (m = 1 or 2 stored vectors, coefficients coef[s ldc + j]), |w|^2 per block
// in part.  Four rows at a time with all their loads (both vectors' planes
// and w) issued together, so a block waits for memory twice instead of once
// per vector and again for w.  Graph mode (dx): vectors x - 1, x.
__global__ void __launch_bounds__(NTHREADS) k_ring_df(float4 *__restrict__ w, const float4 *__restrict__ V, uint64_t D,
                                                      int j0, int m, const double2 *__restrict__ coef, int ldc,
                                                      const SecView *__restrict__ secs,
                                                      const int *__restrict__ chunk0, int S,
                                                      const int *__restrict__ active, double2 *__restrict__ part,
                                                      const int *__restrict__ dx = nullptr) {
    if (dx) {
        graph_range(dx, 1, j0, m);
        coef += j0;
    }
    __shared__ float4 cf[2];
    __shared__ double red[NTHREADS / 32];
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    if (threadIdx.x < 2)
        cf[threadIdx.x] = threadIdx.x < m ? split2(coef[(uint64_t)ci.s * ldc + threadIdx.x]) : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const float4 c0 = cf[0], c1 = cf[1];
    const float2 *h0 = (const float2 *)(V + (uint64_t)j0 * D), *l0 = h0 + D;
    const float2 *h1 = m > 1 ? (const float2 *)(V + (uint64_t)(j0 + 1) * D) : h0, *l1 = h1 + D;
    const int nk = (ci.n - (int)threadIdx.x + NTHREADS - 1) / NTHREADS;
    const uint64_t r0 = ci.base + threadIdx.x;
    dfl n2 = {0.f, 0.f};
#pragma unroll
    for (int kb = 0; kb < RPT; kb += 4) {
        float2 a0h[4], a0l[4], a1h[4], a1l[4];
        float4 wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t r = r0 + (uint64_t)(kb + u) * NTHREADS;
            if (kb + u < nk) {
                a0h[u] = h0[r];
                a0l[u] = l0[r];
                a1h[u] = h1[r];
                a1l[u] = l1[r];
                wv[u] = w[r];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (kb + u >= nk) continue;
            dfl ur = {0.f, 0.f}, ui = {0.f, 0.f};
            // u = c0 v0 + c1 v1: re += a.r c.r - a.i c.i ; im += a.r c.i + a.i c.r
            df_mac(ur, a0h[u].x, a0l[u].x, c0.x, c0.y);
            df_mac(ur, -a0h[u].y, -a0l[u].y, c0.z, c0.w);
            df_mac(ui, a0h[u].x, a0l[u].x, c0.z, c0.w);
            df_mac(ui, a0h[u].y, a0l[u].y, c0.x, c0.y);
            if (m > 1) {
                df_mac(ur, a1h[u].x, a1l[u].x, c1.x, c1.y);
                df_mac(ur, -a1h[u].y, -a1l[u].y, c1.z, c1.w);
                df_mac(ui, a1h[u].x, a1l[u].x, c1.z, c1.w);
                df_mac(ui, a1h[u].y, a1l[u].y, c1.x, c1.y);
            }
            const dfl re = df_sum({wv[u].x, wv[u].y}, {-ur.hi, -ur.lo});
            const dfl im = df_sum({wv[u].z, wv[u].w}, {-ui.hi, -ui.lo});
            w[r0 + (uint64_t)(kb + u) * NTHREADS] = make_float4(re.hi, re.lo, im.hi, im.lo);
            df_mac(n2, re.hi, re.lo, re.hi, re.lo);
            df_mac(n2, im.hi, im.lo, im.hi, im.lo);
        }
    }
    double nrm = df_d(n2);
#pragma unroll
    for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < NTHREADS / 32; ++q) t += red[q];
        part[blockIdx.x] = make_double2(t, 0.0);
    }
}

// double-float engine: basis vector x + 1 = w * inv[s], all in double-float
// (the store's slot x + 1, and hin, the interleaved input of the next H Phi)
__global__ void __launch_bounds__(NTHREADS) k_scale_df(const float4 *__restrict__ w, float4 *__restrict__ out,
                                                       float4 *__restrict__ hin, const double *__restrict__ inv,
                                                       const SecView *__restrict__ secs,
                                                       const int *__restrict__ chunk0, int S,
                                                       const int *__restrict__ active,
                                                       const int *__restrict__ dx, uint64_t D) {
    if (dx) out += (uint64_t)(*dx + 1) * D;     // graph mode: out is the store's base, vector x + 1
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const float2 fs = split_d(inv[ci.s]);
    const dfl f = {fs.x, fs.y};
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            const float4 v = w[ci.base + r];
            const dfl re = df_mul({v.x, v.y}, f), im = df_mul({v.z, v.w}, f);
            const float4 q = make_float4(re.hi, re.lo, im.hi, im.lo);
            st_st(out, D, ci.base + r, q);
            hin[ci.base + r] = q;
        }
    }
}

// element r of an output vector starting at p (slot length D for the store)
__device__ __forceinline__ void st_comb(double *p, uint64_t, uint64_t r, dfl re, dfl) {
    p[r] = (double)re.hi + (double)re.lo;
}
__device__ __forceinline__ void st_comb(double2 *p, uint64_t, uint64_t r, dfl re, dfl im) {
    p[r] = make_double2((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo);
}
__device__ __forceinline__ void st_comb(float2 *p, uint64_t D, uint64_t r, dfl re, dfl) {
    re = df_norm(re);
    st_st(p, D, r, make_float4(re.hi, re.lo, 0.f, 0.f));
}
__device__ __forceinline__ void st_comb(float4 *p, uint64_t D, uint64_t r, dfl re, dfl im) {
    re = df_norm(re);
    im = df_norm(im);
    st_st(p, D, r, make_float4(re.hi, re.lo, im.hi, im.lo));
}

// out_y[r] = sum_x V_x[r] C[s][x][y] (y < nout <= 16) over a double-float
// basis, for the rows of sectors with mask[s] != 0; OT is fp64 (a result) or
// the double-float store itself (the thick restart)
template <typename VT, typename OT>
__global__ void __launch_bounds__(NTHREADS) k_combine_df(OT *__restrict__ out, uint64_t ldo,
                                                         const typename DfS<VT>::T *__restrict__ V, uint64_t D,
                                                         int nin, int nout, const double *__restrict__ C, int ldc,
                                                         const SecView *__restrict__ secs,
                                                         const int *__restrict__ chunk0, int S,
                                                         const int *__restrict__ mask) {
    extern __shared__ float2 scc[];
    __shared__ int nx;
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (mask && !mask[ci.s]) return;
    const double *Cs = C + (uint64_t)ci.s * ldc;
    if (threadIdx.x == 0) nx = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nin * nout; i += blockDim.x) {
        scc[i] = split_d(Cs[i]);
        if (Cs[i] != 0.0) atomicMax(&nx, i / nout + 1);
    }
    __syncthreads();
    nin = nx;      // vectors past the sector's last nonzero coefficient may be unwritten
#pragma unroll 1
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r >= ci.n) continue;
        dfl re[MAXOUT], im[MAXOUT];
#pragma unroll
        for (int y = 0; y < MAXOUT; ++y) re[y] = im[y] = {0.f, 0.f};
#pragma unroll 4
        for (int x = 0; x < nin; ++x) {
            const float4 a = ld_st(V + (uint64_t)x * D, D, ci.base + r);
#pragma unroll
            for (int y = 0; y < MAXOUT; ++y)
                if (y < nout) {
                    const float2 c = scc[x * nout + y];
                    df_mac(re[y], a.x, a.y, c.x, c.y);
                    if (IsC<VT>::v) df_mac(im[y], a.z, a.w, c.x, c.y);
                }
        }
#pragma unroll
        for (int y = 0; y < MAXOUT; ++y)
            if (y < nout) st_comb(out + (uint64_t)y * ldo, ldo, ci.base + r, re[y], im[y]);
    }
}

// one output vector (nout = 1, the Lanczos Ritz vector): out[r] = sum_x V_x[r]
// C[s][x], double-float accumulation, each thread's RPT rows in registers so
// every pass over a stored vector has all of a thread's loads in flight.
// DFS: the store is double-float (slots of D elements, see ld_st); else the
// fp32 vectors of the fp32 engine.
__device__ __forceinline__ float4 ld_comb(const float *p) { return make_float4(*p, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 ld_comb(const float2 *p) { const float2 v = *p; return make_float4(v.x, 0.f, v.y, 0.f); }
template <typename VT, typename SV, typename OT, bool DFS>
__global__ void __launch_bounds__(NTHREADS) k_combine1(OT *__restrict__ out, uint64_t ldo, const SV *__restrict__ V,
                                                       uint64_t D, int nin, const double *__restrict__ C, int ldc,
                                                       const SecView *__restrict__ secs,
                                                       const int *__restrict__ chunk0, int S,
                                                       const int *__restrict__ mask) {
    extern __shared__ float2 scc[];
    __shared__ int nx;
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (mask && !mask[ci.s]) return;
    const double *Cs = C + (uint64_t)ci.s * ldc;
    if (threadIdx.x == 0) nx = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nin; i += blockDim.x) {
        scc[i] = split_d(Cs[i]);
        if (Cs[i] != 0.0) atomicMax(&nx, i + 1);
    }
    __syncthreads();
    nin = nx;      // vectors past the sector's last nonzero coefficient may be unwritten
    dfl re[RPT], im[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) re[k] = im[k] = {0.f, 0.f};
    for (int x = 0; x < nin; ++x) {
        const float2 c = scc[x];
        const SV *slot = V + (uint64_t)x * D;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = threadIdx.x + k * NTHREADS;
            if (r < ci.n) {
                float4 a;
                if constexpr (DFS) a = ld_st(slot, D, ci.base + r);
                else a = ld_comb(slot + ci.base + r);
                df_mac(re[k], a.x, a.y, c.x, c.y);
                if (IsC<VT>::v) df_mac(im[k], a.z, a.w, c.x, c.y);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) st_comb(out, ldo, ci.base + r, re[k], im[k]);
    }
}

// part[c] = sum |t - e_s v|^2 (residual of an eigenpair)
template <typename WT>
__global__ void __launch_bounds__(NTHREADS) k_resid(const WT *__restrict__ t, const WT *__restrict__ v,
                                                    const double *__restrict__ e, const SecView *__restrict__ secs,
                                                    const int *__restrict__ chunk0, int S, double2 *__restrict__ part) {
    __shared__ double red[NTHREADS / 32];
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    const double es = e[ci.s];
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r < ci.n) {
            const double2 a = ld2(t + ci.base + r), b = ld2(v + ci.base + r);
            const double dx = a.x - es * b.x, dy = a.y - es * b.y;
            acc += dx * dx + dy * dy;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < NTHREADS / 32; ++q) s += red[q];
        part[blockIdx.x] = make_double2(s, 0.0);
    }
}

// ----------------------------------------------------- small host eigensolvers

// cyclic Jacobi for a dense symmetric n x n matrix (row-major A, destroyed);
// eigenvalues ascending in w, eigenvectors in the columns of Z (row-major)
static void jacobi_eig(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &Z) {
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {       // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {       // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {       // Z <- Z J
                    const double zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
                    Z[(size_t)k * n + p] = c * zkp - s * zkq;
                    Z[(size_t)k * n + q] = s * zkp + c * zkq;
                }
            }
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return A[(size_t)x * n + x] < A[(size_t)y * n + y]; });
    w.resize(n);
    std::vector<double> Z2((size_t)n * n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[(size_t)ord[j] * n + ord[j]];
        for (int i = 0; i < n; ++i) Z2[(size_t)i * n + j] = Z[(size_t)i * n + ord[j]];
    }
    Z.swap(Z2);
}

// ------------------------------------------------------------------- engine

// QS3_LOG=1 in the environment prints one line per convergence check to stderr
static bool log_on() {
    static int v = -1;
    if (v < 0) { const char *e = getenv("QS3_LOG"); v = (e && *e && *e != '0') ? 1 : 0; }
    return v == 1;
}

// H Phi work and device time of a solve: CUDA events around every H Phi
// launch on the solve's stream, read back at the solver's sync points
struct HphiStats {
    uint64_t nnz = 0;
    double sec = 0.0;
    int calls = 0;
    int graph_calls = 0;                  // calls replayed inside CUDA graphs (not in sec)
    // the Gram-Schmidt dot-product pass (outside graphs): device time, launches,
    // algorithmic bytes (stored vectors read + w read)
    double gs_sec = 0.0;
    int gs_calls = 0;
    uint64_t gs_bytes = 0;
    uint64_t gs_fma = 0;                  // binary64 FMAs of those launches (binary64 engine)
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pend, pend_gs, freel;
    ~HphiStats() {
        for (auto &p : pend) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
        for (auto &p : pend_gs) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
        for (auto &p : freel) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    }
    int pair(std::pair<cudaEvent_t, cudaEvent_t> &p) {
        if (!freel.empty()) { p = freel.back(); freel.pop_back(); return QS3_OK; }
        QS3_CUDA(cudaEventCreate(&p.first));
        QS3_CUDA(cudaEventCreate(&p.second));
        return QS3_OK;
    }
    // call after the stream has been synchronised
    int harvest() {
        for (auto &p : pend) {
            float ms = 0.f;
            QS3_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
            sec += 1e-3 * ms;
            freel.push_back(p);
        }
        pend.clear();
        for (auto &p : pend_gs) {
            float ms = 0.f;
            QS3_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
            gs_sec += 1e-3 * ms;
            freel.push_back(p);
        }
        pend_gs.clear();
        return QS3_OK;
    }
};

template <typename VT>
struct Engine {
    using WT = typename Wide<VT>::T;       // fp64 vector type of the same kind
    using ST = typename DfS<VT>::T;        // storage type of the Krylov basis
    static constexpr bool DF = Is64<VT>::v;
    Basis &B;
    cudaStream_t st;
    HphiStats *stats;
    int cap = 0, nscr = 0;
    uint64_t D = 0;
    DevBuf V, ring, part, h1, h2, alpha, beta, nrm, nrm1, inv, active;
    int rp = 0, rc = 1, rw = 2;           // fp64 ring: psi_{x-1}, psi_x, work (DF only)
    std::vector<int> h_active;
    double brk;
    // CUDA graphs (DF engine): one captured step per ring phase (indexed by
    // rc); its kernels take the step index x from device memory (xdev)
    bool graphs = false;
    DevBuf xdev;
    int xdev_val = -1;                    // value the device holds after the work queued so far
    cudaStream_t cs = nullptr;            // capture stream
    cudaGraphExec_t gx[3] = {nullptr, nullptr, nullptr};
    long long gnodes[3] = {0, 0, 0};

    Engine(Basis &b, cudaStream_t s, HphiStats *hs) : B(b), st(s), stats(hs) { brk = DF ? 1e-12 : 1e-6; }
    ~Engine() {
        for (auto &g : gx)
            if (g) cudaGraphExecDestroy(g);
        if (cs) cudaStreamDestroy(cs);
    }
    Engine(const Engine &) = delete;
    Engine &operator=(const Engine &) = delete;
    // double-float engine (fp64 complex k-sector solves; set before init):
    // H is applied to the stored double-float psi_x (QS3_C128DF) and w = H
    // psi_x, its three-term and Gram-Schmidt updates and the scaling into
    // psi_{x+1} all stay in double-float (float4 per element, wdf) on the
    // fp32 units; the fp64 ring then only carries the start vector
    bool dfh = false;
    DevBuf wdf, hdf;                      // w, and the interleaved copy of psi_x that H reads
    float4 *wd() { return wdf.as<float4>(); }
    float4 *hd() { return hdf.as<float4>(); }
    void use_df_hphi(bool on) { dfh = on && DF && IsC<VT>::v && B.has_k && B.nd > 0; }
    void set_strict(bool) {}
    // the whole Lanczos loop as one graph: the double-float engine, whose
    // step does not rotate a host-side ring
    bool loop_graph_ok() const { return graphs && dfh; }
    // replay Lanczos steps as CUDA graphs (fp64 engine; ignored otherwise)
    int enable_graphs(bool on) {
        graphs = on && DF && B.nchunks > 0;
        if (graphs && !xdev.p) QS3_TRY(xdev.alloc(sizeof(int)));
        return QS3_OK;
    }

    qs3_dtype dtype() const {
        if (sizeof(VT) == 4) return QS3_F32;
        if (sizeof(VT) == 8) return DF ? QS3_F64 : QS3_C64;
        return QS3_C128;
    }
    // stored basis vector j (slots cap .. cap + nscr - 1 are scratch)
    ST *svec(int j) { return V.as<ST>() + (uint64_t)j * D; }
    VT *rvec(int i) { return ring.as<VT>() + (uint64_t)i * D; }
    // the vector H is applied to at step x, and where H psi_x goes
    VT *hin(int x) {
        if constexpr (DF) return rvec(rc); else return svec(x);
    }
    VT *hout(int x) {
        if constexpr (DF) return rvec(rw); else return svec(x + 1);
    }
    const SecView *secs() { return B.d_secs.as<SecView>(); }
    const int *c0() { return B.d_chunk0.as<int>(); }
    int *act() { return active.as<int>(); }

    int init(int cap_, int nscratch) {
        cap = cap_;
        nscr = nscratch;
        D = B.total;
        QS3_TRY(V.alloc((uint64_t)(cap + nscr) * D * sizeof(ST)));
        if (DF) QS3_TRY(ring.alloc(3 * D * sizeof(VT)));
        if (dfh) {
            QS3_TRY(wdf.alloc(D * sizeof(float4)));
            QS3_TRY(hdf.alloc(D * sizeof(float4)));
            QS3_CUDA(cudaMemsetAsync(wdf.p, 0, wdf.n, st));
        }
        QS3_TRY(part.alloc((uint64_t)std::max(B.nchunks, 1) * cap * sizeof(double2)));
        QS3_TRY(h1.alloc((uint64_t)B.S * cap * sizeof(double2)));
        QS3_TRY(h2.alloc((uint64_t)B.S * cap * sizeof(double2)));
        QS3_TRY(alpha.alloc((uint64_t)B.S * cap * sizeof(double)));
        QS3_TRY(beta.alloc((uint64_t)B.S * cap * sizeof(double)));
        QS3_TRY(nrm.alloc((uint64_t)B.S * sizeof(double2)));
        QS3_TRY(nrm1.alloc((uint64_t)B.S * sizeof(double2)));
        QS3_TRY(inv.alloc((uint64_t)B.S * sizeof(double)));
        QS3_TRY(active.alloc((uint64_t)B.S * sizeof(int)));
        QS3_CUDA(cudaMemsetAsync(alpha.p, 0, alpha.n, st));
        QS3_CUDA(cudaMemsetAsync(beta.p, 0, beta.n, st));
        h_active.assign(B.S, 0);
        for (int s = 0; s < B.S; ++s) h_active[s] = B.dims[s] > 0;
        QS3_TRY(push_active());
        return tune_dots();
    }
    int check_err() { return QS3_OK; }     // no bounded device waits here
    int push_active() {
        QS3_CUDA(cudaMemcpyAsync(active.p, h_active.data(), B.S * sizeof(int), cudaMemcpyHostToDevice, st));
        return QS3_OK;
    }
    bool any_active() const {
        for (int a : h_active) if (a) return true;
        return false;
    }
    int grid() const { return std::max(B.nchunks, 1); }

    // reduce part[.. m] into out (S x ldo)
    int reduce(int m, double2 *out, int ldo, bool df = false) {
        dim3 g(m, B.S);
        if (df) k_reduce_df<<<dim3((m + 7) / 8, B.S), NTHREADS, 0, st>>>((const float4 *)part.p, m, c0(), act(), out, ldo);
        else k_reduce<<<g, NTHREADS, 0, st>>>(part.as<double2>(), m, c0(), act(), out, ldo);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    // dot products / update against the stored basis vectors j0 .. j0 + m - 1
    // (w: VT, or float4 for the double-float engine)
    template <typename WV>
    int mdot(int j0, int m, const WV *w, double2 *out, int ldo) {
        if (B.nchunks == 0) return QS3_OK;
        QS3_TRY(mdot_df(B.tune_nv, j0, m, w, nullptr));
        return reduce(m, out, ldo, true);
    }
    // k_mdot_df with nv basis vectors per pass (1, 2 or 4; other values: 2);
    // graph mode (dx): ring selects the three-term range (see graph_range)
    template <typename WV>
    int mdot_df(int nv, int j0, int m, const WV *w, const int *dx, int ring = 0) {
        {
            const ST *v = V.as<ST>();
            float4 *pp = (float4 *)part.p;
            if (ring || (!dx && m <= 2)) nv = std::min(nv, 2);      // the three-term pass: 2 vectors
            if (nv == 1)
                k_mdot_df<VT, 1, WV><<<grid(), NTHREADS, 0, st>>>(v, D, j0, m, w, secs(), c0(), B.S, act(), pp, dx, ring);
            else if (nv == 4)
                k_mdot_df<VT, 4, WV><<<grid(), NTHREADS, 0, st>>>(v, D, j0, m, w, secs(), c0(), B.S, act(), pp, dx, ring);
            else
                k_mdot_df<VT, 2, WV><<<grid(), NTHREADS, 0, st>>>(v, D, j0, m, w, secs(), c0(), B.S, act(), pp, dx, ring);
            QS3_LAUNCHED();
        }
        return QS3_OK;
    }
    // autotuner for the staging depth of the dot products: time 1, 2 and 4
    // vectors per pass on min(cap, 48) stored vectors (their contents do not
    // matter for the timing; the partial sums are discarded) and keep the
    // fastest for this basis
    int tune_dots() {
        if constexpr (DF) {
            if (B.tune_nv != 0 || B.nchunks == 0) return QS3_OK;
            cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
            QS3_CUDA(cudaStreamIsCapturing(st, &cst));
            if (cst != cudaStreamCaptureStatusNone) return QS3_OK;
            const int m = std::min(cap, 48);
            cudaEvent_t e0, e1;
            QS3_CUDA(cudaEventCreate(&e0));
            QS3_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            int bnv = 2;
            int rc2 = QS3_OK;
            for (int nv : {1, 2, 4}) {
                float tmin = 1e30f;
                for (int rep = 0; rep < 4 && rc2 == QS3_OK; ++rep) {
                    if (cudaEventRecord(e0, st) != cudaSuccess) { rc2 = QS3_ERR_CUDA; break; }
                    rc2 = dfh ? mdot_df(nv, 0, m, (const float4 *)wd(), nullptr)
                              : mdot_df(nv, 0, m, (const VT *)rvec(rw), nullptr);
                    if (rc2 != QS3_OK) break;
                    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                        rc2 = QS3_ERR_CUDA;
                        break;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) tmin = std::min(tmin, ms);     // the first run warms up
                }
                if (tmin < best) { best = tmin; bnv = nv; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc2 != QS3_OK) return set_err(rc2, "dot-product autotuning failed");
            B.tune_nv = bnv;
        }
        return QS3_OK;
    }
    // nrm_out (optional): per-sector |w|^2 after the update; wn2 (DF, optional):
    // |w|^2 before it, which lets small-coefficient updates run in plain fp32
    template <typename WV>
    int mupdate(WV *w, int j0, int m, const double2 *cf, int ldc, double2 *nrm_out, const double2 *wn2 = nullptr) {
        if (B.nchunks == 0) return QS3_OK;
        double2 *pp = nrm_out ? part.as<double2>() : nullptr;
        if constexpr (DF)
            k_mupdate_df<VT, WV><<<grid(), NTHREADS, m * sizeof(float4), st>>>(w, V.as<ST>(), D, j0, m, cf, ldc, secs(),
                                                                             c0(), B.S, act(), wn2, pp);
        else
            k_mupdate32<VT><<<grid(), NTHREADS, m * sizeof(float4), st>>>((VT *)w, V.as<VT>(), D, j0, m, cf, ldc, secs(),
                                                                          c0(), B.S, act(), pp);
        QS3_LAUNCHED();
        if (nrm_out) return reduce(1, nrm_out, 1);
        return QS3_OK;
    }
    // the same against the exact fp64 psi_{x-1}, psi_x of the ring (DF only);
    // h gets the coefficients at h + j0, j0 = max(0, x - 1); n2 the new |w|^2
    int ring_pass(int x, VT *w, double2 *h, double2 *n2) {
        if (B.nchunks == 0) return QS3_OK;
        const int m = x > 0 ? 2 : 1;
        const VT *v0 = x > 0 ? rvec(rp) : rvec(rc);
        const int64_t ld = (int64_t)(rvec(rc) - rvec(rp));
        const int j0 = std::max(0, x - 1);
        if constexpr (DF) {
            k_mdot<VT><<<grid(), NTHREADS, 0, st>>>(v0, ld, 0, m, w, secs(), c0(), B.S, act(), part.as<double2>());
            QS3_LAUNCHED();
            QS3_TRY(reduce(m, h + j0, cap));
            k_mupdate<VT><<<grid(), NTHREADS, m * sizeof(double2), st>>>(w, v0, ld, 0, m, h + j0, cap, secs(), c0(), B.S,
                                                                        act(), part.as<double2>());
            QS3_LAUNCHED();
            QS3_TRY(reduce(1, n2, 1));
        }
        return QS3_OK;
    }
    // scale w by inv per sector; DF: also store its double-float copy as basis vector j
    int scale_store(VT *w, int j) {
        if (B.nchunks == 0) return QS3_OK;
        if constexpr (DF)
            k_scale_split<VT><<<grid(), NTHREADS, 0, st>>>(w, svec(j), inv.as<double>(), secs(), c0(), B.S, act(),
                                                           nullptr, D, dfh ? hd() : nullptr);
        else
            k_scale<VT><<<grid(), NTHREADS, 0, st>>>(w, inv.as<double>(), secs(), c0(), B.S, act());
        QS3_LAUNCHED();
        return QS3_OK;
    }
    // normalise the start vector hin(0) per sector (and store it as basis vector 0)
    int normalise_start() {
        if (B.nchunks == 0) return QS3_OK;
        k_norm2<VT><<<grid(), NTHREADS, 0, st>>>(hin(0), secs(), c0(), B.S, act(), part.as<double2>());
        QS3_LAUNCHED();
        QS3_TRY(reduce(1, nrm.as<double2>(), 1));
        k_inv_sqrt<<<(B.S + 127) / 128, 128, 0, st>>>(B.S, nrm.as<double2>(), inv.as<double>());
        QS3_LAUNCHED();
        return scale_store(hin(0), 0);
    }
    int start_random(uint64_t seed) {
        if (B.nchunks == 0) return QS3_OK;
        k_random<VT><<<grid(), NTHREADS, 0, st>>>(hin(0), seed, secs(), c0(), B.S);
        QS3_LAUNCHED();
        return normalise_start();
    }
    int start_from(const WT *src) {
        if (B.nchunks == 0) return QS3_OK;
        k_convert<VT, WT><<<grid(), NTHREADS, 0, st>>>(hin(0), src, secs(), c0(), B.S, nullptr);
        QS3_LAUNCHED();
        return normalise_start();
    }
    // one step on stream st with every x-dependent count and offset taken
    // from xdev (the body of the captured graphs; DF engine, not full2)
    int step_body_dev() {
        const int *dx = xdev.as<int>();
        if constexpr (DF) {
            if (dfh) return step_body_dev_df(dx);
        }
        VT *w = rvec(rw);
        QS3_TRY(hphi_launch(B, dtype(), rvec(rc), w, st, act()));
        const int64_t ld = (int64_t)(rvec(rc) - rvec(rp));
        double2 *hh1 = h1.as<double2>(), *n1 = nrm1.as<double2>();
        if constexpr (DF) {
            k_mdot<VT><<<grid(), NTHREADS, 0, st>>>(rvec(rp), ld, 0, 2, w, secs(), c0(), B.S, act(), part.as<double2>(),
                                                    dx);
            QS3_LAUNCHED();
            k_reduce<<<dim3(2, B.S), NTHREADS, 0, st>>>(part.as<double2>(), 2, c0(), act(), hh1, cap, dx, true);
            QS3_LAUNCHED();
            k_mupdate<VT><<<grid(), NTHREADS, 2 * sizeof(double2), st>>>(w, rvec(rp), ld, 0, 2, hh1, cap, secs(), c0(),
                                                                        B.S, act(), part.as<double2>(), dx);
            QS3_LAUNCHED();
            k_reduce<<<dim3(1, B.S), NTHREADS, 0, st>>>(part.as<double2>(), 1, c0(), act(), n1, 1);
            QS3_LAUNCHED();
            QS3_TRY(mdot_df(B.tune_nv, 0, cap, w, dx));
            k_reduce_df<<<dim3(std::min((cap + 7) / 8, 8), B.S), NTHREADS, 0, st>>>((const float4 *)part.p, cap, c0(), act(),
                                                                           h2.as<double2>(), cap, dx);
            QS3_LAUNCHED();
            k_mupdate_df<VT><<<grid(), NTHREADS, cap * sizeof(float4), st>>>(w, V.as<ST>(), D, 0, cap, h2.as<double2>(),
                                                                           cap, secs(), c0(), B.S, act(), n1,
                                                                           part.as<double2>(), dx);
            QS3_LAUNCHED();
            k_reduce<<<dim3(1, B.S), NTHREADS, 0, st>>>(part.as<double2>(), 1, c0(), act(), nrm.as<double2>(), 1);
            QS3_LAUNCHED();
            k_step_scalars<<<(B.S + 127) / 128, 128, 0, st>>>(B.S, 0, cap, hh1, nrm.as<double2>(), act(),
                                                             alpha.as<double>(), beta.as<double>(), inv.as<double>(),
                                                             brk, dx);
            QS3_LAUNCHED();
            k_scale_split<VT><<<grid(), NTHREADS, 0, st>>>(w, V.as<ST>(), inv.as<double>(), secs(), c0(), B.S, act(), dx,
                                                           D);
            QS3_LAUNCHED();
            k_advance<<<1, 1, 0, st>>>(xdev.as<int>());
            QS3_LAUNCHED();
        }
        return QS3_OK;
    }
    // the double-float engine's step with x from xdev (x >= 1)
    int step_body_dev_df(const int *dx) {
        float4 *w = wd();
        const ST *v = V.as<ST>();
        double2 *hh1 = h1.as<double2>(), *n1 = nrm1.as<double2>();
        QS3_TRY(hphi_df_launch(B, hd(), nullptr, 0, w, st, act(), true));
        // three-term part against psi_{x-1}, psi_x
        QS3_TRY(mdot_df(B.tune_nv, 0, 2, (const float4 *)w, dx, 1));
        k_reduce_df<<<dim3(1, B.S), NTHREADS, 0, st>>>((const float4 *)part.p, 2, c0(), act(), hh1, cap, dx, 1);
        QS3_LAUNCHED();
        k_ring_df<<<grid(), NTHREADS, 0, st>>>(w, V.as<float4>(), D, 0, 2, hh1, cap, secs(), c0(), B.S, act(),
                                               part.as<double2>(), dx);
        QS3_LAUNCHED();
        k_reduce<<<dim3(1, B.S), NTHREADS, 0, st>>>(part.as<double2>(), 1, c0(), act(), n1, 1);
        QS3_LAUNCHED();
        // one Gram-Schmidt pass against psi_0 .. psi_x
        QS3_TRY(mdot_df(B.tune_nv, 0, cap, (const float4 *)w, dx, 0));
        k_reduce_df<<<dim3(std::min((cap + 7) / 8, 8), B.S), NTHREADS, 0, st>>>((const float4 *)part.p, cap, c0(), act(),
                                                                       h2.as<double2>(), cap, dx, 0);
        QS3_LAUNCHED();
        k_mupdate_df<VT, float4><<<grid(), NTHREADS, cap * sizeof(float4), st>>>(w, v, D, 0, cap, h2.as<double2>(), cap,
                                                                                secs(), c0(), B.S, act(), n1,
                                                                                part.as<double2>(), dx, 0);
        QS3_LAUNCHED();
        k_reduce<<<dim3(1, B.S), NTHREADS, 0, st>>>(part.as<double2>(), 1, c0(), act(), nrm.as<double2>(), 1);
        QS3_LAUNCHED();
        k_step_scalars<<<(B.S + 127) / 128, 128, 0, st>>>(B.S, 0, cap, hh1, nrm.as<double2>(), act(), alpha.as<double>(),
                                                         beta.as<double>(), inv.as<double>(), brk, dx);
        QS3_LAUNCHED();
        k_scale_df<<<grid(), NTHREADS, 0, st>>>(w, V.as<float4>(), hd(), inv.as<double>(), secs(), c0(), B.S, act(),
                                                dx, D);
        QS3_LAUNCHED();
        k_advance<<<1, 1, 0, st>>>(xdev.as<int>());
        QS3_LAUNCHED();
        return QS3_OK;
    }
    // the graph of the current ring phase (one graph for the double-float
    // engine, whose step does not rotate the ring), captured on first use
    int graph_step(int x) {
        if (!cs) QS3_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const int gi = dfh ? 0 : rc;
        if (!gx[gi]) {
            cudaStream_t keep = st;
            st = cs;
            cudaGraph_t g = nullptr;
            QS3_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            const int r = step_body_dev();
            const cudaError_t e = cudaStreamEndCapture(cs, &g);
            st = keep;
            if (r != QS3_OK) {
                if (g) cudaGraphDestroy(g);
                return r;
            }
            if (e != cudaSuccess) return set_err(QS3_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            const cudaError_t ei = cudaGraphInstantiate(&gx[gi], g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                gx[gi] = nullptr;
                return set_err(QS3_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
            }
            gnodes[gi] = (long long)nn;
            count_launch(-(long long)nn);   // the capture ran nothing
        }
        if (xdev_val != x) {
            k_setx<<<1, 1, 0, st>>>(xdev.as<int>(), x);
            QS3_LAUNCHED();
        }
        QS3_CUDA(cudaGraphLaunch(gx[gi], st));
        count_launch(gnodes[gi]);
        xdev_val = x + 1;
        return QS3_OK;
    }
    // Alg. 10 lines 5-11 for step x: psi_{x+1} from H psi_x
    // full2: two Gram-Schmidt passes against all of psi_0..psi_x (the first
    // step after a thick restart, where v also has the large arrowhead
    // components beta_y psi_y).  Otherwise the large components of v lie
    // along psi_{x-1}, psi_x only: they are removed first (the three-term
    // recurrence, coefficients by dot product), then one classical
    // Gram-Schmidt pass against every kept vector removes the O(eps) rest.
    int step(int x, bool full2 = false) {
        if (DF && graphs && !full2 && x >= 1) {
            // H Phi inside a graph is not timed separately
            stats->calls += 1;
            stats->graph_calls += 1;
            for (int s = 0; s < B.S; ++s)
                if (h_active[s]) stats->nnz += B.nnz_sec[s];
            QS3_TRY(graph_step(x));
            if (!dfh) {
                const int o = rp;
                rp = rc;
                rc = rw;
                rw = o;
            }
            return QS3_OK;
        }
        if constexpr (DF) {
            if (dfh) return step_df(x, full2);
        }
        VT *w = hout(x);
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        QS3_TRY(stats->pair(ev));
        QS3_CUDA(cudaEventRecord(ev.first, st));
        QS3_TRY(hphi_launch(B, dtype(), hin(x), w, st, act()));
        QS3_CUDA(cudaEventRecord(ev.second, st));
        stats->pend.push_back(ev);
        stats->calls += 1;
        for (int s = 0; s < B.S; ++s)
            if (h_active[s]) stats->nnz += B.nnz_sec[s];
        const int j0 = full2 ? 0 : std::max(0, x - 1);
        double2 *n1 = DF ? nrm1.as<double2>() : nullptr;
        if (DF && !full2) {
            QS3_TRY(ring_pass(x, w, h1.as<double2>(), n1));
        } else {
            QS3_TRY(mdot(j0, x + 1 - j0, w, h1.as<double2>() + j0, cap));
            QS3_TRY(mupdate(w, j0, x + 1 - j0, h1.as<double2>() + j0, cap, n1));
        }
        QS3_TRY(gs_dots(x, (const VT *)w, h2.as<double2>()));
        QS3_TRY(mupdate(w, 0, x + 1, h2.as<double2>(), cap, nrm.as<double2>(), n1));
        k_step_scalars<<<(B.S + 127) / 128, 128, 0, st>>>(B.S, x, cap, h1.as<double2>(), nrm.as<double2>(), act(),
                                                         alpha.as<double>(), beta.as<double>(), inv.as<double>(), brk);
        QS3_LAUNCHED();
        QS3_TRY(scale_store(w, x + 1));
        if (DF) {                            // psi_{x+1} becomes the current ring vector
            const int o = rp;
            rp = rc;
            rc = rw;
            rw = o;
        }
        return QS3_OK;
    }
    // the double-float engine's step (see dfh)
    int step_df(int x, bool full2) {
        float4 *w = wd();
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        QS3_TRY(stats->pair(ev));
        QS3_CUDA(cudaEventRecord(ev.first, st));
        QS3_TRY(hphi_df_launch(B, hd(), nullptr, 0, w, st, act(), true));
        QS3_CUDA(cudaEventRecord(ev.second, st));
        stats->pend.push_back(ev);
        stats->calls += 1;
        for (int s = 0; s < B.S; ++s)
            if (h_active[s]) stats->nnz += B.nnz_sec[s];
        // three-term part (full2: all of psi_0 .. psi_x), then one Gram-Schmidt pass
        const int j0 = full2 ? 0 : std::max(0, x - 1);
        double2 *n1 = nrm1.as<double2>();
        QS3_TRY(mdot(j0, x + 1 - j0, (const float4 *)w, h1.as<double2>() + j0, cap));
        if (full2 || B.nchunks == 0) {
            QS3_TRY(mupdate(w, j0, x + 1 - j0, h1.as<double2>() + j0, cap, n1));
        } else if constexpr (std::is_same<ST, float4>::value) {
            k_ring_df<<<grid(), NTHREADS, 0, st>>>(w, V.as<float4>(), D, j0, x + 1 - j0, h1.as<double2>() + j0, cap,
                                                   secs(), c0(), B.S, act(), part.as<double2>());
            QS3_LAUNCHED();
            QS3_TRY(reduce(1, n1, 1));
        }
        QS3_TRY(gs_dots(x, (const float4 *)w, h2.as<double2>()));
        QS3_TRY(mupdate(w, 0, x + 1, h2.as<double2>(), cap, nrm.as<double2>(), n1));
        k_step_scalars<<<(B.S + 127) / 128, 128, 0, st>>>(B.S, x, cap, h1.as<double2>(), nrm.as<double2>(), act(),
                                                         alpha.as<double>(), beta.as<double>(), inv.as<double>(), brk);
        QS3_LAUNCHED();
        if constexpr (std::is_same<ST, float4>::value) {
            if (B.nchunks > 0) {
                k_scale_df<<<grid(), NTHREADS, 0, st>>>(w, svec(x + 1), hd(), inv.as<double>(), secs(), c0(), B.S,
                                                        act(), nullptr, D);
                QS3_LAUNCHED();
            }
        }
        return QS3_OK;
    }
    // the Gram-Schmidt dot pass against psi_0 .. psi_x, timed with events
    template <typename WV>
    int gs_dots(int x, const WV *w, double2 *out) {
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        QS3_TRY(stats->pair(ev));
        QS3_CUDA(cudaEventRecord(ev.first, st));
        QS3_TRY(mdot(0, x + 1, w, out, cap));
        QS3_CUDA(cudaEventRecord(ev.second, st));
        stats->pend_gs.push_back(ev);
        stats->gs_calls += 1;
        uint64_t rows = 0;
        for (int s = 0; s < B.S; ++s)
            if (h_active[s]) rows += B.dims[s];
        stats->gs_bytes += rows * ((uint64_t)(x + 1) * sizeof(ST) + sizeof(WV));
        return QS3_OK;
    }
    int fetch(std::vector<double> &a, std::vector<double> &b) {
        a.resize((size_t)B.S * cap);
        b.resize((size_t)B.S * cap);
        QS3_CUDA(cudaMemcpyAsync(a.data(), alpha.p, a.size() * 8, cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaMemcpyAsync(b.data(), beta.p, b.size() * 8, cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaStreamSynchronize(st));
        return stats->harvest();
    }
    // out_y = sum_x psi_x C[s][x][y] (x < nin) for sectors with mask; C host,
    // S x (nin*nout); OT is WT (a result) or ST (into the scratch slots)
    template <typename OT>
    int combine(OT *out, uint64_t ldo, int nin, int nout, const std::vector<double> &C, const std::vector<int> &mask) {
        if (B.nchunks == 0) return QS3_OK;
        if (nout > MAXOUT) return set_err(QS3_ERR_INVALID_ARG, "at most %d vectors per combination", MAXOUT);
        const int ldc = nin * nout;
        DevBuf dC, dm;
        QS3_TRY(dC.alloc(C.size() * 8));
        QS3_TRY(dm.alloc(mask.size() * 4));
        QS3_CUDA(cudaMemcpyAsync(dC.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, st));
        QS3_CUDA(cudaMemcpyAsync(dm.p, mask.data(), mask.size() * 4, cudaMemcpyHostToDevice, st));
        // one fp64 result, or one double-float stored vector
        constexpr bool one_ok = DF || std::is_same<OT, WT>::value;
        if (one_ok && nout == 1) {
            if constexpr (one_ok)
                k_combine1<VT, ST, OT, DF><<<grid(), NTHREADS, ldc * sizeof(float2), st>>>(out, ldo, V.as<ST>(), D, nin,
                                                                                          dC.as<double>(), ldc, secs(),
                                                                                          c0(), B.S, dm.as<int>());
        } else if constexpr (DF)
            k_combine_df<VT, OT><<<grid(), NTHREADS, ldc * sizeof(float2), st>>>(out, ldo, V.as<ST>(), D, nin, nout,
                                                                                 dC.as<double>(), ldc, secs(), c0(),
                                                                                 B.S, dm.as<int>());
        else
            k_combine<VT, OT><<<grid(), NTHREADS, ldc * sizeof(double), st>>>(out, ldo, V.as<VT>(), D, nin, nout,
                                                                              dC.as<double>(), ldc, secs(), c0(), B.S,
                                                                              dm.as<int>());
        QS3_LAUNCHED();
        QS3_CUDA(cudaStreamSynchronize(st));     // dC/dm are released on return
        return QS3_OK;
    }
    // thick restart (Alg. 10 lines 14-19): psi_y = Psi C[:, y] for y < NK
    // (through the scratch slots), psi_NK = psi_NM (the fp64 ring of a DF
    // engine, or H's double-float input, already holds psi_NM)
    int thick_restart(int NM, int NK, const std::vector<double> &C) {
        QS3_TRY(combine<ST>(svec(cap), B.total, NM, NK, C, h_active));
        QS3_CUDA(cudaMemcpyAsync(svec(0), svec(cap), (size_t)NK * B.total * sizeof(ST), cudaMemcpyDeviceToDevice, st));
        QS3_CUDA(cudaMemcpyAsync(svec(NK), svec(NM), (size_t)B.total * sizeof(ST), cudaMemcpyDeviceToDevice, st));
        return QS3_OK;
    }
};

}  // namespace qs3

#include "qs3_engine64.cuh"

namespace qs3 {

// residual |H v - e v| of fp64 vectors (one per sector, concatenated); returns max over sectors
template <typename WT>
static int residuals(Basis &B, const WT *v, const std::vector<double> &e, cudaStream_t st, double &rmax,
                     std::vector<double> *per = nullptr) {
    rmax = 0.0;
    if (B.nchunks == 0) return QS3_OK;
    DevBuf t, de, part, out;
    QS3_TRY(t.alloc(B.total * sizeof(WT)));
    QS3_TRY(de.alloc(B.S * 8));
    QS3_TRY(part.alloc((uint64_t)B.nchunks * sizeof(double2)));
    QS3_TRY(out.alloc(B.S * sizeof(double2)));
    QS3_CUDA(cudaMemcpyAsync(de.p, e.data(), B.S * 8, cudaMemcpyHostToDevice, st));
    const qs3_dtype dt = sizeof(WT) == 8 ? QS3_F64 : QS3_C128;
    QS3_TRY(hphi_launch(B, dt, v, t.p, st, nullptr));
    k_resid<WT><<<B.nchunks, NTHREADS, 0, st>>>(t.as<WT>(), v, de.as<double>(), B.d_secs.as<SecView>(),
                                                B.d_chunk0.as<int>(), B.S, part.as<double2>());
    QS3_LAUNCHED();
    dim3 g(1, B.S);
    k_reduce<<<g, NTHREADS, 0, st>>>(part.as<double2>(), 1, B.d_chunk0.as<int>(), nullptr, out.as<double2>(), 1);
    QS3_LAUNCHED();
    std::vector<double2> h(B.S);
    QS3_CUDA(cudaMemcpyAsync(h.data(), out.p, B.S * sizeof(double2), cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaStreamSynchronize(st));
    if (per) per->assign(B.S, 0.0);
    for (int s = 0; s < B.S; ++s) {
        if (!B.dims[s]) continue;
        const double r = std::sqrt(std::max(h[s].x, 0.0));
        rmax = std::max(rmax, r);
        if (per) (*per)[s] = r;
    }
    return QS3_OK;
}

// ------------------------------------------------------- conventional Lanczos
// The convergence checks of Alg. 10 (the lowest Ritz value of the
// tridiagonal T_m and its Ritz residual, the small eigenproblem K8) run on
// the device, one warp per sector, so the loop needs no host round trip: the
// step kernels and the check form the body of a CUDA graph WHILE node whose
// condition the device sets (graph mode), or the host launches them and
// reads one flag every check_every steps (direct mode).  Both run the same
// kernels, so their results are identical.

// number of eigenvalues of the symmetric tridiagonal (a, b) below x: the sign
// changes of the Sturm sequence p_0 = 1, p_i = (a_{i-1} - x) p_{i-1} -
// b_{i-2}^2 p_{i-2} (the leading principal minors of T - x I).  No division:
// p_i and p_{i-1} are rescaled together by a power of two when |p_i| leaves
// [2^-500, 2^500], which keeps every ratio exact.  A vanishing p_i takes the
// sign opposite to p_{i-1} (one change, as for a zero pivot of T - x I = L D L^T
// counted negative).
__device__ int sturm_count_dev(int n, const double *__restrict__ a, const double *__restrict__ bb, double x) {
    // bb[i] = b_{i-1}^2 (bb[0] unused).  Signs, zeros and the rescaling test
    // read the bit pattern in integer instructions, so the only fp64 work on
    // the dependent chain is the fma of each step.
    int cnt = 0, sp = 1;
    double pm = 0.0, p = 1.0;
    for (int i = 0; i < n; ++i) {
        const double t = i ? bb[i] * pm : 0.0;
        const double pn = fma(a[i] - x, p, -t);
        const long long bits = __double_as_longlong(pn);
        const bool zero = (bits << 1) == 0;
        const int sn = zero ? -sp : (bits < 0 ? -1 : 1);
        cnt += sn != sp;
        sp = sn;
        pm = p;
        p = pn;
        const int e = (int)((bits >> 52) & 0x7ff);
        if (e > 1523 || (e < 523 && !zero)) {        // |p| >= 2^501 or 0 < |p| < 2^-500
            const double f = e > 1523 ? 0x1p-500 : 0x1p500;
            p *= f;
            pm *= f;
        }
    }
    return cnt;
}

// lowest eigenvalue of the tridiagonal of order n by multisection: the warp
// evaluates the Sturm count at 31 interior points of a bracket and keeps
// the first sub-interval that holds an eigenvalue, until the bracket stops
// shrinking in fp64 (all lanes return the same value).  The bracket starts
// around e_prev when given (the lowest Ritz value of a shorter Krylov space,
// which the new one does not exceed) and falls back to the Gershgorin bounds.
__device__ double tri_lowest_warp(int n, const double *__restrict__ a, const double *__restrict__ b,
                                  const double *__restrict__ bb, double e_prev) {
    const int lane = threadIdx.x & 31;
    double lo = 1e300, hi = -1e300;
    for (int i = lane; i < n; i += 32) {
        const double r = (i ? fabs(b[i - 1]) : 0.0) + (i < n - 1 ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double w = fmax(hi - lo, 1e-300);
    lo -= 1e-3 * w;
    hi += 1e-3 * w;
    if (isfinite(e_prev) && e_prev > lo && e_prev < hi) {
        // lane 0 tests e_prev + margin (an eigenvalue lies below it), lanes
        // 1..31 a ladder below e_prev at distances 1e-6 w 4^-(lane-1): the
        // Ritz value moved down by a small, shrinking amount since e_prev,
        // so the last ladder point without an eigenvalue below it and the
        // first with one bracket it to within a factor of four of that move
        const double t = lane == 0 ? e_prev + 1e-12 * w : e_prev - ldexp(1e-6 * w, -2 * (lane - 1));
        const int c = sturm_count_dev(n, a, bb, t);
        const unsigned some = __ballot_sync(0xffffffffu, lane > 0 && c > 0);   // counts rise with t
        const unsigned none = __ballot_sync(0xffffffffu, lane > 0 && c == 0);
        const int c0 = __shfl_sync(0xffffffffu, c, 0);
        const double t0 = __shfl_sync(0xffffffffu, t, 0);
        if (c0 > 0 && t0 < hi) hi = t0;
        if (none) {
            const int jl = 31 - __clz(none);                                    // the highest point with none
            const double tl = __shfl_sync(0xffffffffu, t, jl);
            if (tl > lo && tl < hi) lo = tl;
        }
        const unsigned above = some & ~((2u << (31 - __clz(none | 1u))) - 1u);
        if (above) {
            const double th = __shfl_sync(0xffffffffu, t, __ffs(above) - 1);   // the lowest point above it with one
            if (th < hi && th > lo) hi = th;
        }
    }
    for (int it = 0; it < 64; ++it) {
        const double h = (hi - lo) / 32.0;
        const double xl = lo + h * (double)(lane + 1);
        const int cnt = (lane < 31 && xl > lo && xl < hi) ? sturm_count_dev(n, a, bb, xl) : 0;
        const unsigned mk = __ballot_sync(0xffffffffu, lane < 31 && cnt > 0);
        const int j = mk ? __ffs(mk) - 1 : 31;
        const double nlo = j == 0 ? lo : fmax(lo, lo + h * (double)j);
        const double nhi = j == 31 ? hi : fmin(hi, lo + h * (double)(j + 1));
        if (!(nlo > lo || nhi < hi)) break;
        lo = nlo;
        hi = nhi;
    }
    return 0.5 * (lo + hi);
}

// eigenvector of the tridiagonal for eigenvalue e by inverse iteration
// (Gaussian elimination with partial pivoting on T - e I; one thread),
// largest component positive; ws holds 5 n doubles of workspace.  From the
// start vector in v (start) and `sweeps` sweeps, else from all ones and
// three sweeps.
__device__ void tri_vec_dev(int n, const double *__restrict__ a, const double *__restrict__ b, double e,
                            double *__restrict__ v, double *__restrict__ ws, bool start = false, int sweeps = 3) {
    if (!start)
        for (int i = 0; i < n; ++i) v[i] = 1.0;
    if (n == 1) {
        v[0] = 1.0;
        return;
    }
    double *d = ws, *du = ws + n, *du2 = ws + 2 * n, *dl = ws + 3 * n, *x = ws + 4 * n;
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(a[i]) + (i < n - 1 ? fabs(b[i]) : 0.0));
    const double pert = fmax(scale, 1e-300) * 1e-14;
    for (int it = 0; it < sweeps; ++it) {
        for (int i = 0; i < n; ++i) {
            d[i] = a[i] - e - pert;
            du[i] = i < n - 1 ? b[i] : 0.0;
            dl[i] = du[i];
            du2[i] = 0.0;
        }
        // x[i] records whether row i was swapped (partial pivoting)
        for (int i = 0; i < n - 1; ++i) {
            if (fabs(d[i]) >= fabs(dl[i])) {
                x[i] = 0.0;
                if (d[i] == 0.0) d[i] = 1e-300;
                const double f = dl[i] / d[i];
                dl[i] = f;
                d[i + 1] -= f * du[i];
            } else {
                x[i] = 1.0;
                const double f = d[i] / dl[i];
                d[i] = dl[i];
                dl[i] = f;
                const double t = du[i];
                du[i] = d[i + 1];
                d[i + 1] = t - f * d[i + 1];
                if (i < n - 2) { du2[i] = du[i + 1]; du[i + 1] = -f * du[i + 1]; }
            }
        }
        if (d[n - 1] == 0.0) d[n - 1] = 1e-300;
        // forward sweep in place in v (the right-hand side)
        for (int i = 0; i < n - 1; ++i) {
            if (x[i] == 0.0) v[i + 1] -= dl[i] * v[i];
            else { const double t = v[i]; v[i] = v[i + 1]; v[i + 1] = t - dl[i] * v[i + 1]; }
        }
        v[n - 1] /= d[n - 1];
        v[n - 2] = (v[n - 2] - du[n - 2] * v[n - 1]) / d[n - 2];
        for (int i = n - 3; i >= 0; --i) v[i] = (v[i] - du[i] * v[i + 1] - du2[i] * v[i + 2]) / d[i];
        double nr = 0.0;
        for (int i = 0; i < n; ++i) nr += v[i] * v[i];
        nr = sqrt(nr);
        if (!(nr > 0.0) || !isfinite(nr)) {
            for (int i = 0; i < n; ++i) v[i] = 1.0;
            break;
        }
        for (int i = 0; i < n; ++i) v[i] /= nr;
    }
    int im = 0;
    for (int i = 1; i < n; ++i) if (fabs(v[i]) > fabs(v[im])) im = i;
    if (v[im] < 0.0) for (int i = 0; i < n; ++i) v[i] = -v[i];
}

// |y_n| of the normalised eigenvector y of the tridiagonal for eigenvalue e,
// for the Ritz residual beta |y_n|: y solved from the bottom up with y_n = 1,
// y_{k-1} = -((a_k - e) y_k + b_k y_{k+1}) / b_{k-1} (rb = 1 / b), then
// normalised.  The lowest Ritz vector of a converging Lanczos run decays
// towards the bottom, so the recurrence follows its growing direction and
// keeps |y_n| to about a percent down to 1e-20 (measured against dense
// eigenvectors), while the forward recurrences lose it below ~1e-8.  Growth
// past 2^500 means |y_n| < 2^-500: returned as 0.  One thread.
__device__ double tri_last_dev(int n, const double *__restrict__ a, const double *__restrict__ b,
                               const double *__restrict__ rb, double e) {
    double yk = 1.0, yk1 = 0.0, nrm = 1.0;
    for (int k = n - 1; k >= 1; --k) {
        const double t = k + 1 < n ? b[k] * yk1 : 0.0;
        const double y = -fma(a[k] - e, yk, t) * rb[k - 1];
        nrm = fma(y, y, nrm);
        yk1 = yk;
        yk = y;
        if (((__double_as_longlong(y) >> 52) & 0x7ff) > 1523) return 0.0;
    }
    return 1.0 / sqrt(nrm);
}

// the bottom-up solution of tri_last_dev stored in v and normalised (its
// entries below 2^-500 of the largest flushed to 0): the start vector of one
// inverse-iteration sweep for the Ritz coefficients, which it leaves as
// accurate as three sweeps from all ones (measured against dense
// eigenvectors).  One thread.
__device__ void tri_bottom_up_dev(int n, const double *__restrict__ a, const double *__restrict__ b,
                                  const double *__restrict__ rb, double e, double *__restrict__ v) {
    v[n - 1] = 1.0;
    for (int k = n - 1; k >= 1; --k) {
        const double t = k + 1 < n ? b[k] * v[k + 1] : 0.0;
        v[k - 1] = -fma(a[k] - e, v[k], t) * rb[k - 1];
        if (((__double_as_longlong(v[k - 1]) >> 52) & 0x7ff) > 1523)
            for (int i = k - 1; i < n; ++i) v[i] *= 0x1p-500;
    }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm = fma(v[i], v[i], nrm);
    const double f = 1.0 / sqrt(nrm);
    for (int i = 0; i < n; ++i) v[i] *= f;
}

// per-sector state of the convergence checks (device)
struct LzState {
    DevBuf eprev, eval, msz, conv, coef, ws, cont, nnz;
    int init(int S, int cap, cudaStream_t st) {
        QS3_TRY(eprev.alloc((size_t)S * 8));
        QS3_TRY(eval.alloc((size_t)S * 8));
        QS3_TRY(msz.alloc((size_t)S * 4));
        QS3_TRY(conv.alloc((size_t)S * 4));
        QS3_TRY(coef.alloc((size_t)S * cap * 8));
        QS3_TRY(ws.alloc((size_t)S * 7 * cap * 8));
        QS3_TRY(cont.alloc(4));
        QS3_TRY(nnz.alloc(8));
        // eprev = NaN (no previous Ritz value); everything else 0
        QS3_CUDA(cudaMemsetAsync(eprev.p, 0xff, eprev.n, st));
        QS3_CUDA(cudaMemsetAsync(eval.p, 0xff, eval.n, st));
        QS3_CUDA(cudaMemsetAsync(msz.p, 0, msz.n, st));
        QS3_CUDA(cudaMemsetAsync(conv.p, 0, conv.n, st));
        QS3_CUDA(cudaMemsetAsync(nnz.p, 0, nnz.n, st));
        return QS3_OK;
    }
};

// after n steps (n = *dx in graph mode): for every active sector count the
// step's H Phi work, and when a check is due (n >= min_iter and n a multiple
// of every, or n = nmax) take the lowest Ritz value e of T_m (m = n, or up
// to the first vanishing beta: an invariant subspace, whose Ritz values are
// exact).  Converged: |e - e_prev| <= eps |e| and the Ritz residual
// beta_{m-1} |c_{m-1}| <= res_tol max(|e|, 1).  A converged sector (or any at
// n = nmax) stores its Ritz coefficients and leaves the active set.
// With lz_smem(cap) bytes of dynamic shared memory the sector's alpha, beta,
// the inverse-iteration workspace, the eigenvector, 1 / beta and beta^2 live
// in shared memory (the dependent stores and loads then stay on the SM; the
// vector is copied to coef at the end); else ws (7 cap per sector) holds the
// workspaces and the rest is read and written in global memory.
__host__ __device__ constexpr size_t lz_smem_need(int cap) { return (size_t)10 * cap * sizeof(double); }
static size_t lz_smem(int cap) { return lz_smem_need(cap) <= 48 * 1024 ? lz_smem_need(cap) : 0; }

__global__ void __launch_bounds__(32) k_lz_check(int n_arg, const int *__restrict__ dx, const double *__restrict__ alpha,
                                                 const double *__restrict__ beta, int cap, int *__restrict__ active,
                                                 const uint64_t *__restrict__ nnz_sec,
                                                 unsigned long long *__restrict__ nnz_acc, double *__restrict__ eprev,
                                                 double *__restrict__ eval, int *__restrict__ msz,
                                                 int *__restrict__ conv, double *__restrict__ coef,
                                                 double *__restrict__ ws, double eps, double res_tol, int min_iter,
                                                 int every, int nmax) {
    extern __shared__ double lzs[];
    const int s = blockIdx.x, lane = threadIdx.x;
    const int n = dx ? *dx : n_arg;
    if (!active[s]) return;
    if (lane == 0) atomicAdd(nnz_acc, (unsigned long long)nnz_sec[s]);
    if (!((n >= min_iter && n % every == 0) || n >= nmax)) return;
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const double *a = alpha + (size_t)s * cap, *b = beta + (size_t)s * cap;
    double *wsp = ws + (size_t)s * 7 * cap;          // inverse-iteration workspace (5 cap), 1 / b, b^2
    double *rb = wsp + 5 * cap, *bb = wsp + 6 * cap;
    double *const vg = coef + (size_t)s * cap;
    double *v = vg;
    const bool sm = dyn >= lz_smem_need(cap);
    if (sm) {
        double *sa = lzs, *sb = lzs + cap;
        for (int i = lane; i < n; i += 32) {
            sa[i] = a[i];
            sb[i] = b[i];
        }
        __syncwarp();
        a = sa;
        b = sb;
        wsp = lzs + 2 * cap;
        v = lzs + 7 * cap;
        rb = lzs + 8 * cap;
        bb = lzs + 9 * cap;
    }
    // the first vanishing beta ends the Krylov sequence
    int m = n;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const unsigned z = __ballot_sync(0xffffffffu, k0 + lane < n && b[k0 + lane] == 0.0);
        if (z) { m = k0 + __ffs(z); break; }
    }
    const bool brk = m < n || b[m - 1] == 0.0;
    for (int i = 1 + lane; i < m; i += 32) bb[i] = b[i - 1] * b[i - 1];
    __syncwarp();
    const double ep = eprev[s];
    const double e = tri_lowest_warp(m, a, b, bb, ep);
    bool ok = brk || (isfinite(ep) && fabs(e - ep) <= eps * fabs(e));
    // the Ritz residual beta_{m-1} |y_m| once the value is stable
    const bool need_res = ok && !brk && res_tol > 0.0;
    if (ok) {
        for (int i = lane; i < m - 1; i += 32) rb[i] = 1.0 / b[i];
        __syncwarp();
    }
    if (need_res) {
        double ym = 0.0;
        if (lane == 0) ym = tri_last_dev(m, a, b, rb, e);
        ym = __shfl_sync(0xffffffffu, ym, 0);
        ok = fabs(b[m - 1]) * ym <= res_tol * fmax(fabs(e), 1.0);
    }
    const bool done = ok || n >= nmax;
    if (lane == 0) {
        eprev[s] = e;
        eval[s] = e;
        msz[s] = m;
        if (done) {
            // the Ritz coefficients of a sector that leaves the active set:
            // converged, one inverse-iteration sweep from the bottom-up
            // solution; stopped at n_max, three sweeps from all ones
            if (ok) {
                tri_bottom_up_dev(m, a, b, rb, e, v);
                tri_vec_dev(m, a, b, e, v, wsp, true, 1);
            } else {
                tri_vec_dev(m, a, b, e, v, wsp);
            }
            conv[s] = ok ? 1 : 0;
            active[s] = 0;
        }
    }
    if (sm && done) {
        __syncwarp();
        for (int i = lane; i < m; i += 32) vg[i] = v[i];
    }
}

// loop condition after n steps: some sector still active and n < nmax;
// written to *cont and, in graph mode, to the WHILE node's condition
__global__ void __launch_bounds__(32) k_lz_cond(int n_arg, const int *__restrict__ dx, const int *__restrict__ active,
                                                int S, int nmax, int *__restrict__ cont,
                                                cudaGraphConditionalHandle h, int use_h) {
    const int n = dx ? *dx : n_arg;
    int any = 0;
    for (int s = threadIdx.x; s < S; s += 32) any |= active[s];
    any = __any_sync(0xffffffffu, any);
    if (threadIdx.x == 0) {
        const int c = (any && n < nmax) ? 1 : 0;
        *cont = c;
        if (use_h) cudaGraphSetConditional(h, c);
    }
}

struct LzResult {
    std::vector<double> e;       // per sector
    std::vector<int> conv;
    int steps = 0;
};

// the Lanczos loop of steps 1 .. (until no sector is active or nmax) as one
// graph: [k_lz_cond -> WHILE { step, k_lz_check, k_lz_cond }], captured once
template <typename EN>
static int lanczos_loop_graph(EN &E, LzState &K, Basis &B, const qs3_solve_opts &o, int nmax, int every,
                              const uint64_t *nnz_sec, int &steps) {
    cudaStream_t cs = nullptr;
    QS3_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t keep = E.st;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    int rc = QS3_OK;
    auto fail = [&](const char *what, cudaError_t e) {
        rc = set_err(QS3_ERR_CUDA, "Lanczos loop graph, %s: %s", what, cudaGetErrorString(e));
    };
    do {
        cudaError_t e;
        if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) { fail("create", e); break; }
        cudaGraphConditionalHandle h;
        if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, 0)) != cudaSuccess) { fail("handle", e); break; }
        // prologue: the first condition
        if ((e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess) { fail("capture", e); break; }
        k_lz_cond<<<1, 32, 0, cs>>>(0, E.xdev.template as<int>(), E.act(), B.S, nmax, K.cont.as<int>(), h, 1);
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess) {
            fail("capture info", e);
            cudaGraph_t tmp;
            cudaStreamEndCapture(cs, &tmp);
            break;
        }
        std::vector<cudaGraphNode_t> dv(deps, deps + nd);
        if ((e = cudaStreamEndCapture(cs, &g)) != cudaSuccess) { fail("end capture", e); break; }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wn;
        if ((e = cudaGraphAddNode(&wn, g, dv.data(), nullptr, dv.size(), &cp)) != cudaSuccess) { fail("while", e); break; }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // body: one step (x from xdev, advanced by the step), the check and the condition
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess) { fail("body capture", e); break; }
        E.st = cs;
        int r = E.step_body_dev();
        if (r == QS3_OK) {
            k_lz_check<<<B.S, 32, lz_smem(E.cap), cs>>>(0, E.xdev.template as<int>(), E.alpha.template as<double>(),
                                           E.beta.template as<double>(), E.cap, E.act(), nnz_sec,
                                           K.nnz.as<unsigned long long>(), K.eprev.as<double>(), K.eval.as<double>(),
                                           K.msz.as<int>(), K.conv.as<int>(), K.coef.as<double>(), K.ws.as<double>(),
                                           o.eps, o.res_tol, o.min_iter, every, nmax);
            k_lz_cond<<<1, 32, 0, cs>>>(0, E.xdev.template as<int>(), E.act(), B.S, nmax, K.cont.as<int>(), h, 1);
        }
        E.st = keep;
        cudaGraph_t bo = nullptr;
        e = cudaStreamEndCapture(cs, &bo);
        if (r != QS3_OK) { rc = r; break; }
        if (e != cudaSuccess) { fail("body end capture", e); break; }
        size_t nn = 0;
        cudaGraphGetNodes(body, nullptr, &nn);
        count_launch(-(long long)(nn - 2));   // the step's kernels were counted while captured
        if ((e = cudaGraphInstantiate(&gx, g, 0)) != cudaSuccess) { gx = nullptr; fail("instantiate", e); break; }
        // x = 1 on the device, then the whole loop
        k_setx<<<1, 1, 0, E.st>>>(E.xdev.template as<int>(), 1);
        count_launch();
        if ((e = cudaGraphLaunch(gx, E.st)) != cudaSuccess) { fail("launch", e); break; }
        if ((e = cudaStreamSynchronize(E.st)) != cudaSuccess) { fail("run", e); break; }
        if ((e = cudaMemcpy(&steps, E.xdev.p, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fail("step count", e);
            break;
        }
        count_launch(1 + (long long)(steps - 1) * (long long)nn);    // the prologue and every iteration
    } while (false);
    if (gx) cudaGraphExecDestroy(gx);
    if (g) cudaGraphDestroy(g);
    if (cs) {
        cudaStreamSynchronize(E.st);
        cudaStreamDestroy(cs);
    }
    return rc;
}

// Lanczos to the lowest eigenpair of each sector; out (fp64, total dim) gets the vectors.
template <typename VT, typename EN = Engine<VT>>
static int lanczos_run(Basis &B, const qs3_solve_opts &o, const typename Wide<VT>::T *start,
                       typename Wide<VT>::T *out, cudaStream_t st, LzResult &R, HphiStats &hs) {
    EN E(B, st, &hs);
    const int nmax = std::max(2, o.n_max);
    E.use_df_hphi(o.hphi_ieee == 0);
    E.set_strict(o.strict64 != 0);
    QS3_TRY(E.init(nmax + 1, 0));
    QS3_TRY(E.enable_graphs(o.use_graphs != 0));
    if (start) QS3_TRY(E.start_from(start)); else QS3_TRY(E.start_random(o.seed));
    const int S = B.S;
    R.e.assign(S, NAN);
    R.conv.assign(S, 0);
    for (int s = 0; s < S; ++s)
        if (!B.dims[s]) R.conv[s] = 1;
    const int every = std::max(1, o.check_every);
    LzState K;
    QS3_TRY(K.init(S, E.cap, st));
    DevBuf dnnz;
    QS3_TRY(dnnz.upload(B.nnz_sec.data(), (size_t)S * 8));
    const uint64_t nz0 = hs.nnz;
    int cont = 0;
    auto check = [&](int n) -> int {
        k_lz_check<<<S, 32, lz_smem(E.cap), st>>>(n, nullptr, E.alpha.template as<double>(), E.beta.template as<double>(), E.cap,
                                     E.act(), dnnz.as<uint64_t>(), K.nnz.as<unsigned long long>(),
                                     K.eprev.as<double>(), K.eval.as<double>(), K.msz.as<int>(), K.conv.as<int>(),
                                     K.coef.as<double>(), K.ws.as<double>(), o.eps, o.res_tol, o.min_iter, every,
                                     nmax);
        QS3_LAUNCHED();
        return QS3_OK;
    };
    auto cond = [&](int n) -> int {
        k_lz_cond<<<1, 32, 0, st>>>(n, nullptr, E.act(), S, nmax, K.cont.as<int>(), 0, 0);
        QS3_LAUNCHED();
        QS3_CUDA(cudaMemcpyAsync(&cont, K.cont.p, 4, cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaStreamSynchronize(st));
        // the host copy of the active set (the engine's statistics)
        QS3_CUDA(cudaMemcpy(E.h_active.data(), E.active.p, S * sizeof(int), cudaMemcpyDeviceToHost));
        return QS3_OK;
    };
    if (B.nchunks > 0) {
        QS3_TRY(E.step(0));
        QS3_TRY(check(1));
        QS3_TRY(cond(1));
        if (cont && E.loop_graph_ok()) {
            QS3_TRY(lanczos_loop_graph(E, K, B, o, nmax, every, dnnz.as<uint64_t>(), R.steps));
            hs.calls += R.steps - 1;
            hs.graph_calls += R.steps - 1;
        } else {
            int x = 1;
            for (; cont && x < nmax; ++x) {
                QS3_TRY(E.step(x));
                const int n = x + 1;
                QS3_TRY(check(n));
                if ((n >= o.min_iter && n % every == 0) || n >= nmax) QS3_TRY(cond(n));
            }
            R.steps = x;
        }
    }
    // results of every sector (the converged ones and those stopped at nmax)
    std::vector<double> ev(S), coef((size_t)S * E.cap);
    std::vector<int> msz(S), conv(S);
    unsigned long long nzd = 0;
    QS3_CUDA(cudaMemcpyAsync(ev.data(), K.eval.p, S * 8, cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaMemcpyAsync(msz.data(), K.msz.p, S * 4, cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaMemcpyAsync(conv.data(), K.conv.p, S * 4, cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaMemcpyAsync(coef.data(), K.coef.p, coef.size() * 8, cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaMemcpyAsync(&nzd, K.nnz.p, 8, cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaStreamSynchronize(st));
    QS3_TRY(E.check_err());
    QS3_TRY(hs.harvest());
    hs.nnz = nz0 + nzd;
    if (log_on())
        for (int s = 0; s < S; ++s)
            fprintf(stderr, "[qs3] lanczos vt=%zu s=%d m=%d e=%.17g conv=%d steps=%d\n", sizeof(VT), s, msz[s], ev[s],
                    conv[s], R.steps);
    std::vector<int> fin(S, 0);
    int nin = 0;
    for (int s = 0; s < S; ++s) {
        if (!B.dims[s]) continue;
        R.e[s] = ev[s];
        R.conv[s] = conv[s];
        fin[s] = msz[s] > 0;
        nin = std::max(nin, msz[s]);
    }
    // psi = sum_x c_x psi_x over the computed vectors (later slots are uninitialised)
    if (nin > 0) {
        std::vector<double> C((size_t)S * nin, 0.0);
        for (int s = 0; s < S; ++s)
            if (fin[s])
                for (int k = 0; k < msz[s]; ++k) C[(size_t)s * nin + k] = coef[(size_t)s * E.cap + k];
        QS3_TRY(E.template combine<typename Wide<VT>::T>(out, B.total, nin, 1, C, fin));
    }
    return QS3_OK;
}

// --------------------------------------------------- thick-restart Lanczos

struct TrlResult {
    std::vector<double> e;       // S x n_eig
    std::vector<int> conv;
    int steps = 0, restarts = 0;
};

template <typename VT, typename EN = Engine<VT>>
static int trl_run(Basis &B, const qs3_solve_opts &o, const typename Wide<VT>::T *start,
                   typename Wide<VT>::T *out, cudaStream_t st, TrlResult &R, HphiStats &hs, int nconv = 0,
                   const std::vector<double> *targets = nullptr) {
    using WT = typename Wide<VT>::T;
    const int S = B.S;
    const int NM = std::max(2, o.n_max);
    const int NK = std::max(1, std::min(o.n_keep, NM - 1));
    const int NE = std::max(1, std::min(o.n_eig, NK));
    if (NK > MAXOUT) return set_err(QS3_ERR_INVALID_ARG, "n_keep %d > %d", NK, MAXOUT);
    EN E(B, st, &hs);
    E.use_df_hphi(o.hphi_ieee == 0);
    E.set_strict(o.strict64 != 0);
    QS3_TRY(E.init(NM + 1, NK));
    QS3_TRY(E.enable_graphs(o.use_graphs != 0));
    if (start) QS3_TRY(E.start_from(start)); else QS3_TRY(E.start_random(o.seed));
    R.e.assign((size_t)S * NE, NAN);
    R.conv.assign(S, 0);
    for (int s = 0; s < S; ++s)
        if (!B.dims[s]) R.conv[s] = 1;
    std::vector<double> a, b;
    std::vector<std::vector<double>> ev(S), Cm(S), eprev(S), bK(S), rres(S);
    // nconv > 0 (the binary64 refinement of an fp32 run): the criterion covers
    // the nconv lowest kept values only, needs their Ritz residuals
    // beta_{N_M} |c_{N_M, y}| <= res_tol max(|e_y|, 1), and needs them to
    // reproduce the fp32 run's values (targets, S x nconv) within fp32
    // accuracy, so a copy of a degenerate level that the single start vector
    // lacks at first is waited for; 0: the paper's criterion over all N_K
    // kept values
    const int ny = nconv > 0 ? std::min(nconv, NK) : NK;
    std::vector<int> msize(S, NM);
    int steps = 0;
    // finish the sectors in `done`: write their NE lowest Ritz vectors
    auto finish = [&](const std::vector<int> &done) -> int {
        bool any = false;
        for (int v : done) any |= v != 0;
        if (!any) return QS3_OK;
        std::vector<double> C((size_t)S * NM * NE, 0.0);     // m <= N_M vectors per sector
        for (int s = 0; s < S; ++s) {
            if (!done[s]) continue;
            const int m = msize[s];
            for (int x = 0; x < m; ++x)
                for (int y = 0; y < NE && y < m; ++y) C[(size_t)s * NM * NE + x * NE + y] = Cm[s][(size_t)x * m + y];
            for (int y = 0; y < NE; ++y) R.e[(size_t)s * NE + y] = y < m ? ev[s][y] : NAN;
        }
        QS3_TRY(E.template combine<WT>(out, B.total, NM, NE, C, done));
        for (int s = 0; s < S; ++s)
            if (done[s]) E.h_active[s] = 0;
        return E.push_active();
    };
    // first part of Alg. 10: N_M Lanczos steps
    for (int x = 0; x < NM; ++x) { QS3_TRY(E.step(x)); ++steps; }
    QS3_TRY(E.fetch(a, b));
    {
        std::vector<int> done(S, 0);
        for (int s = 0; s < S; ++s) {
            if (!E.h_active[s]) continue;
            const double *as = &a[(size_t)s * E.cap], *bs = &b[(size_t)s * E.cap];
            int m = NM;
            for (int k = 0; k < NM - 1; ++k)
                if (bs[k] == 0.0) { m = k + 1; break; }
            msize[s] = m;
            std::vector<double> T((size_t)m * m, 0.0);
            for (int i = 0; i < m; ++i) {
                T[(size_t)i * m + i] = as[i];
                if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = bs[i];
            }
            jacobi_eig(m, T, ev[s], Cm[s]);
            rres[s].assign(m, 0.0);
            for (int y = 0; y < m; ++y) rres[s][y] = std::fabs(bs[m - 1] * Cm[s][(size_t)(m - 1) * m + y]);
            if (m < NM || bs[NM - 1] == 0.0) { done[s] = 1; R.conv[s] = 1; }   // Krylov space exhausted
        }
        QS3_TRY(finish(done));
    }
    int I = 1;
    for (; I <= o.max_iter && E.any_active(); ++I) {
        std::vector<int> done(S, 0);
        bool anyc = false;
        for (int s = 0; s < S; ++s) {
            if (!E.h_active[s]) continue;
            if (I > 1) {
                double dmax = 0.0;
                for (int y = 0; y < ny; ++y) dmax = std::max(dmax, std::fabs(eprev[s][y] / ev[s][y] - 1.0));
                bool ok = dmax < o.eps;
                if (ok && nconv > 0 && o.res_tol > 0)
                    for (int y = 0; y < ny && y < (int)rres[s].size(); ++y)
                        ok = ok && rres[s][y] <= o.res_tol * std::max(std::fabs(ev[s][y]), 1.0);
                if (ok && nconv > 0 && targets)
                    for (int y = 0; y < ny; ++y) {
                        const double tg = (*targets)[(size_t)s * ny + y];
                        if (std::isfinite(tg)) ok = ok && std::fabs(ev[s][y] - tg) <= 1e-4 * std::max(std::fabs(tg), 1.0);
                    }
                if (ok) { done[s] = 1; R.conv[s] = 1; anyc = true; }
            }
            eprev[s].assign(ev[s].begin(), ev[s].begin() + NK);
        }
        if (anyc) QS3_TRY(finish(done));
        if (!E.any_active()) break;
        // restart (lines 14-19): psi_y = Psi C[:, y] for y < N_K; psi_{N_K} = psi_{N_M}
        std::vector<double> C((size_t)S * NM * NK, 0.0);
        for (int s = 0; s < S; ++s) {
            if (!E.h_active[s]) continue;
            bK[s].assign(NK, 0.0);
            const double bNM = b[(size_t)s * E.cap + NM - 1];
            for (int y = 0; y < NK; ++y) bK[s][y] = bNM * Cm[s][(size_t)(NM - 1) * NM + y];
            for (int x = 0; x < NM; ++x)
                for (int y = 0; y < NK; ++y) C[(size_t)s * NM * NK + x * NK + y] = Cm[s][(size_t)x * NM + y];
        }
        QS3_TRY(E.thick_restart(NM, NK, C));
        // lines 20-26: Lanczos steps from psi_{N_K} (the Gram-Schmidt against psi_0..psi_{N_K}
        // removes the arrowhead couplings beta_y psi_y)
        for (int x = NK; x < NM; ++x) { QS3_TRY(E.step(x, x == NK)); ++steps; }
        QS3_TRY(E.fetch(a, b));
        // lines 27-30: arrowhead T and its eigen-decomposition
        for (int s = 0; s < S; ++s) {
            if (!E.h_active[s]) continue;
            const double *as = &a[(size_t)s * E.cap], *bs = &b[(size_t)s * E.cap];
            int m = NM;
            for (int k = NK; k < NM - 1; ++k)
                if (bs[k] == 0.0) { m = k + 1; break; }
            std::vector<double> T((size_t)m * m, 0.0);
            for (int y = 0; y < NK; ++y) {
                T[(size_t)y * m + y] = ev[s][y];
                T[(size_t)y * m + NK] = T[(size_t)NK * m + y] = bK[s][y];
            }
            for (int x = NK; x < m; ++x) {
                T[(size_t)x * m + x] = as[x];
                if (x + 1 < m) T[(size_t)x * m + x + 1] = T[(size_t)(x + 1) * m + x] = bs[x];
            }
            std::vector<double> w2, Z2;
            jacobi_eig(m, T, w2, Z2);
            rres[s].assign(m, 0.0);
            for (int y = 0; y < m; ++y) rres[s][y] = std::fabs(bs[m - 1] * Z2[(size_t)(m - 1) * m + y]);
            if (m < NM) {            // invariant subspace: the Ritz values are exact
                msize[s] = m;
                ev[s] = w2;
                Cm[s] = Z2;
                std::vector<int> d1(S, 0);
                d1[s] = 1;
                R.conv[s] = 1;
                QS3_TRY(finish(d1));
                continue;
            }
            ev[s] = w2;
            Cm[s] = Z2;
        }
        R.restarts = I;
    }
    // sectors still running: return their current Ritz pairs
    {
        std::vector<int> rest(S, 0);
        for (int s = 0; s < S; ++s) rest[s] = E.h_active[s];
        QS3_TRY(finish(rest));
    }
    R.steps = steps;
    return E.check_err();
}

// ------------------------------------------------------------- entry points

static bool all_conv(const std::vector<int> &c) {
    for (int v : c) if (!v) return false;
    return true;
}

template <typename V32, typename V64>
static int lanczos_entry(Basis &B, const qs3_solve_opts &o, double *evals, void *evecs, qs3_solve_info *info,
                         cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    uint64_t nz = 0;
    QS3_TRY(count_nnz(B, &nz));
    HphiStats hs;
    DevBuf own;
    V64 *out = (V64 *)evecs;
    if (!out) {
        QS3_TRY(own.alloc(B.total * sizeof(V64)));
        out = own.as<V64>();
    }
    QS3_CUDA(cudaMemsetAsync(out, 0, B.total * sizeof(V64), st));
    LzResult R;
    int iters = 0, refine = 0;
    if (o.precision == QS3_F32) {
        // the fp32 phase stops at fp32 resolution; the fp64 refinement takes it from there
        qs3_solve_opts o1 = o;
        o1.eps = std::max(o.eps, 2e-7);
        o1.res_tol = o.res_tol > 0 ? std::max(o.res_tol, 1e-5) : 0.0;
        QS3_TRY(lanczos_run<V32>(B, o1, nullptr, out, st, R, hs));
        iters += R.steps;
        // fp64 refinement from the fp32 Ritz vector, until the Ritz value is
        // stable to refine_tol (or eps) and the caller's residual test holds
        qs3_solve_opts o2 = o;
        o2.min_iter = std::max(2, std::min(o.min_iter, o.check_every));
        if (o.refine_tol > 0) o2.eps = std::max(o.eps, 0.1 * o.refine_tol);
        LzResult R2;
        QS3_TRY((lanczos_run<V64, Engine64<V64>>(B, o2, out, out, st, R2, hs)));
        refine = R2.steps;
        iters += R2.steps;
        R = R2;
    } else {
        // QS3_F64: the IEEE binary64 engine; QS3_C128DF: the double-float engine
        if (o.precision == QS3_C128DF) QS3_TRY((lanczos_run<V64, Engine<V64>>(B, o, nullptr, out, st, R, hs)));
        else QS3_TRY((lanczos_run<V64, Engine64<V64>>(B, o, nullptr, out, st, R, hs)));
        iters += R.steps;
    }
    for (int s = 0; s < B.S; ++s) evals[s] = R.e[s];
    double rmax = 0.0;
    QS3_TRY(residuals<V64>(B, out, R.e, st, rmax));
    if (info) {
        info->iterations = iters;
        info->restarts = 0;
        int c = 0;
        for (int v : R.conv) c += v;
        info->converged = c;
        info->refine_iterations = refine;
        info->max_residual = rmax;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        QS3_CUDA(cudaStreamSynchronize(st));
        QS3_TRY(hs.harvest());
        info->hphi_nnz = hs.nnz;
        info->hphi_seconds = hs.sec;
        info->hphi_calls = hs.calls;
        info->hphi_graph_calls = hs.graph_calls;
        info->gs_dot_seconds = hs.gs_sec;
        info->gs_dot_bytes = hs.gs_bytes;
        info->gs_dot_calls = hs.gs_calls;
        info->gs_dot_fma = hs.gs_fma;
    }
    return all_conv(R.conv) ? QS3_OK : set_err(QS3_ERR_NOT_CONVERGED, "Lanczos did not converge in %d steps", o.n_max);
}

template <typename V32, typename V64>
static int trl_entry(Basis &B, const qs3_solve_opts &o, double *evals, void *evecs, qs3_solve_info *info,
                     cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    uint64_t nz = 0;
    QS3_TRY(count_nnz(B, &nz));
    HphiStats hs;
    const int NM = std::max(2, o.n_max);
    const int NK = std::max(1, std::min(o.n_keep, NM - 1));
    const int NE = std::max(1, std::min(o.n_eig, NK));
    if (o.n_eig > NK) return set_err(QS3_ERR_INVALID_ARG, "n_eig %d > n_keep %d", o.n_eig, NK);
    DevBuf own;
    V64 *out = (V64 *)evecs;
    if (!out) {
        QS3_TRY(own.alloc((uint64_t)NE * B.total * sizeof(V64)));
        out = own.as<V64>();
    }
    QS3_CUDA(cudaMemsetAsync(out, 0, (uint64_t)NE * B.total * sizeof(V64), st));
    TrlResult R;
    int iters = 0, refine = 0, restarts = 0;
    if (o.precision == QS3_F32) {
        // fp32 phase to fp32 resolution, keeping all N_K Ritz vectors: the
        // criterion covers the N_K kept values, so the fp64 refinement starts
        // from the sum of all of them (its first Krylov space then holds the
        // whole kept set, not only the wanted n_eig)
        qs3_solve_opts o1 = o;
        o1.eps = std::max(o.eps, 2e-7);
        o1.n_eig = NK;
        DevBuf kept;
        QS3_TRY(kept.alloc((uint64_t)NK * B.total * sizeof(V64)));
        QS3_CUDA(cudaMemsetAsync(kept.p, 0, (uint64_t)NK * B.total * sizeof(V64), st));
        QS3_TRY(trl_run<V32>(B, o1, nullptr, kept.as<V64>(), st, R, hs));
        iters += R.steps;
        restarts += R.restarts;
        DevBuf sum;
        QS3_TRY(sum.alloc(B.total * sizeof(V64)));
        {
            std::vector<double> C((size_t)B.S * NK, 1.0);
            std::vector<int> all(B.S, 1);
            DevBuf dC, dm;
            QS3_TRY(dC.alloc(C.size() * 8));
            QS3_TRY(dm.alloc(all.size() * 4));
            QS3_CUDA(cudaMemcpyAsync(dC.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, st));
            QS3_CUDA(cudaMemcpyAsync(dm.p, all.data(), all.size() * 4, cudaMemcpyHostToDevice, st));
            if (B.nchunks) {
                k_combine<V64, V64><<<B.nchunks, NTHREADS, NK * sizeof(double), st>>>(
                    sum.as<V64>(), B.total, kept.as<V64>(), B.total, NK, 1, dC.as<double>(), NK,
                    B.d_secs.as<SecView>(), B.d_chunk0.as<int>(), B.S, dm.as<int>());
                QS3_LAUNCHED();
            }
            QS3_CUDA(cudaStreamSynchronize(st));
        }
        // binary64 refinement: the wanted n_eig values to refine_tol, with
        // their Ritz residuals below refine_tol |E| as well
        TrlResult R2;
        qs3_solve_opts o2 = o;
        if (o.refine_tol > 0) {
            o2.eps = std::max(o.eps, 0.1 * o.refine_tol);
            o2.res_tol = o.refine_tol;
        }
        std::vector<double> tg((size_t)B.S * NE);
        for (int s = 0; s < B.S; ++s)
            for (int y = 0; y < NE; ++y) tg[(size_t)s * NE + y] = R.e[(size_t)s * NK + y];
        QS3_TRY((trl_run<V64, Engine64<V64>>(B, o2, sum.as<V64>(), out, st, R2, hs, NE, &tg)));
        refine = R2.steps;
        iters += R2.steps;
        restarts += R2.restarts;
        R = R2;
    } else {
        if (o.precision == QS3_C128DF) QS3_TRY((trl_run<V64, Engine<V64>>(B, o, nullptr, out, st, R, hs)));
        else QS3_TRY((trl_run<V64, Engine64<V64>>(B, o, nullptr, out, st, R, hs)));
        iters += R.steps;
        restarts += R.restarts;
    }
    for (size_t i = 0; i < R.e.size(); ++i) evals[i] = R.e[i];
    double rmax = 0.0;
    for (int y = 0; y < NE; ++y) {
        std::vector<double> ey(B.S);
        for (int s = 0; s < B.S; ++s) ey[s] = std::isfinite(R.e[(size_t)s * NE + y]) ? R.e[(size_t)s * NE + y] : 0.0;
        double r = 0.0;
        QS3_TRY(residuals<V64>(B, out + (uint64_t)y * B.total, ey, st, r));
        rmax = std::max(rmax, r);
    }
    if (info) {
        info->iterations = iters;
        info->restarts = restarts;
        int c = 0;
        for (int v : R.conv) c += v;
        info->converged = c;
        info->refine_iterations = refine;
        info->max_residual = rmax;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        QS3_CUDA(cudaStreamSynchronize(st));
        QS3_TRY(hs.harvest());
        info->hphi_nnz = hs.nnz;
        info->hphi_seconds = hs.sec;
        info->hphi_calls = hs.calls;
        info->hphi_graph_calls = hs.graph_calls;
        info->gs_dot_seconds = hs.gs_sec;
        info->gs_dot_bytes = hs.gs_bytes;
        info->gs_dot_calls = hs.gs_calls;
        info->gs_dot_fma = hs.gs_fma;
    }
    return all_conv(R.conv) ? QS3_OK
                            : set_err(QS3_ERR_NOT_CONVERGED, "thick-restart Lanczos did not converge in %d restarts",
                                      o.max_iter);
}

static int check_opts(const qs3_solve_opts *o) {
    if (!o) return set_err(QS3_ERR_INVALID_ARG, "options are NULL");
    if (o->n_max < 2 || o->n_max > 2048) return set_err(QS3_ERR_INVALID_ARG, "n_max %d outside [2, 2048]", o->n_max);
    if (o->check_every < 1) return set_err(QS3_ERR_INVALID_ARG, "check_every %d", o->check_every);
    if (!(o->eps > 0)) return set_err(QS3_ERR_INVALID_ARG, "eps %g", o->eps);
    if (o->precision != QS3_F32 && o->precision != QS3_F64 && o->precision != QS3_C128DF)
        return set_err(QS3_ERR_INVALID_ARG, "precision %d", o->precision);
    return QS3_OK;
}

// ---------------------------------------------- Gram-Schmidt dot products
// the dot kernels of the binary64 engine on caller vectors: each V_j copied
// into a word-planar slot, then k_dotx (mode 0) or k_dot64 (mode 1)
template <typename VT>
__global__ void k_to_planar(const VT *__restrict__ x, typename PlS<VT>::T *__restrict__ slot, uint64_t D) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < D; r += (uint64_t)gridDim.x * blockDim.x)
        pl_st(slot, D, r, ld2(x + r));
}

template <typename VT>
static int gs_dots_run(Basis &B, int m, const VT *V, uint64_t ldv, const VT *w, double *out, int mode,
                       cudaStream_t st) {
    using T = typename PlS<VT>::T;
    const uint64_t D = B.total;
    memset(out, 0, (size_t)B.S * m * 2 * sizeof(double));
    if (m == 0 || B.nchunks == 0) return QS3_OK;
    DevBuf pl, dgt, get, part, res, dsl, pr, derr;
    QS3_TRY(pl.alloc((uint64_t)m * D * sizeof(VT)));
    QS3_TRY(part.alloc((uint64_t)B.nchunks * m * (mode == 0 ? XW * 3 * sizeof(long long) : sizeof(double2))));
    QS3_TRY(res.alloc((uint64_t)B.S * m * sizeof(double2)));
    const int g = (int)std::min<uint64_t>((D + 255) / 256, 4096);
    for (int j = 0; j < m; ++j) {
        k_to_planar<VT><<<g, 256, 0, st>>>(V + (uint64_t)j * ldv, pl.as<T>() + (uint64_t)j * 2 * D, D);
        QS3_LAUNCHED();
    }
    const SecView *secs = B.d_secs.as<SecView>();
    const int *c0 = B.d_chunk0.as<int>();
    if (mode == 0) {
        using G = typename DigT<VT>::T;
        QS3_TRY(dgt.alloc((uint64_t)m * D * sizeof(VT) + 16));      // k_dotb reads up to 16 bytes past
        QS3_TRY(get.alloc((uint64_t)m * B.nchunks * XW * sizeof(int)));
        QS3_TRY(derr.alloc(sizeof(int)));
        QS3_CUDA(cudaMemsetAsync(derr.p, 0, sizeof(int), st));
        QS3_TRY(dotb_prepare<VT>());
        k_digitize<VT><<<dim3(B.nchunks, m), XT, 0, st>>>(pl.as<T>(), D, 0, dgt.as<G>(), get.as<int>(), B.nchunks,
                                                           secs, c0, B.S);
        QS3_LAUNCHED();
        QS3_TRY(dotx_launch<VT>(B.tune_nv64 > 0 ? B.tune_nv64 : 2, dgt.as<G>(), get.as<int>(), B.nchunks, D, 0, m,
                                w, secs, c0, B.S, nullptr, part.as<long long>(), st, nullptr, 0, derr.as<int>()));
        const std::vector<int> s0 = reduce_slices(B);
        QS3_TRY(dsl.upload(s0.data(), s0.size() * sizeof(int)));
        QS3_TRY(pr.alloc((uint64_t)std::max(s0[B.S], 1) * m * 5 * sizeof(long long)));
        QS3_TRY(reducex_launch(part.as<long long>(), pr.as<long long>(), m, m, c0, dsl.as<int>(), s0[B.S], B.S,
                               nullptr, res.as<double2>(), m, st, nullptr, 0, IsC<VT>::v ? 1 : 0, one_slice(s0)));
    } else {
        k_dot64<VT, 2><<<B.nchunks, NTHREADS, 0, st>>>(pl.as<T>(), D, 0, m, w, secs, c0, B.S, nullptr,
                                                        part.as<double2>());
        QS3_LAUNCHED();
        k_reduce64<<<dim3((m + 7) / 8, B.S), NTHREADS, 0, st>>>(part.as<double2>(), m, c0, nullptr,
                                                                res.as<double2>(), m);
        QS3_LAUNCHED();
    }
    QS3_CUDA(cudaMemcpyAsync(out, res.p, (size_t)B.S * m * sizeof(double2), cudaMemcpyDeviceToHost, st));
    int e = 0;
    if (derr.p) QS3_CUDA(cudaMemcpyAsync(&e, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaStreamSynchronize(st));
    if (e) return set_err(QS3_ERR_TIMEOUT, "a wait of the dot pass (k_dotb) ran out");
    return QS3_OK;
}

}  // namespace qs3

using namespace qs3;

extern "C" int qs3_lanczos(qs3_basis_t b, const qs3_solve_opts *o, double *evals, void *evecs, qs3_solve_info *info,
                           void *stream) {
    clear_err();
    if (!b || !evals) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    QS3_TRY(check_opts(o));
    if (info) memset(info, 0, sizeof(*info));
    Basis &B = b->B;
    cudaStream_t st = (cudaStream_t)stream;
    if (B.has_k) return lanczos_entry<float2, double2>(B, *o, evals, evecs, info, st);
    return lanczos_entry<float, double>(B, *o, evals, evecs, info, st);
}

extern "C" int qs3_trlanczos(qs3_basis_t b, const qs3_solve_opts *o, double *evals, void *evecs, qs3_solve_info *info,
                             void *stream) {
    clear_err();
    if (!b || !evals) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    QS3_TRY(check_opts(o));
    if (o->n_keep < 1 || o->n_keep >= o->n_max || o->n_keep > MAXOUT)
        return set_err(QS3_ERR_INVALID_ARG, "n_keep %d (need 1 <= n_keep < n_max, n_keep <= %d)", o->n_keep, MAXOUT);
    if (o->n_eig < 1 || o->n_eig > o->n_keep) return set_err(QS3_ERR_INVALID_ARG, "n_eig %d", o->n_eig);
    if (info) memset(info, 0, sizeof(*info));
    Basis &B = b->B;
    cudaStream_t st = (cudaStream_t)stream;
    if (B.has_k) return trl_entry<float2, double2>(B, *o, evals, evecs, info, st);
    return trl_entry<float, double>(B, *o, evals, evecs, info, st);
}

namespace qs3 {

// qs3_hphi with QS3_C128X: phi's digit image (the layout of the engine's
// digit store, one slot) in scratch, then the product
int hphi_x_binary64(Basis &B, const void *phi, void *psi, cudaStream_t st) {
    if (!hphi_x_ok(B))
        return set_err(QS3_ERR_STATE, "QS3_C128X needs a k-sector basis with the representative table and one hop "
                                      "amplitude");
    const uint64_t D = B.total;
    DevBuf pl, dgt, get;
    QS3_TRY(pl.alloc(D * sizeof(double2)));
    QS3_TRY(dgt.alloc(D * sizeof(double2)));
    QS3_TRY(get.alloc((uint64_t)B.nchunks * XW * sizeof(int)));
    const int g = (int)std::min<uint64_t>((D + 255) / 256, 4096);
    k_to_planar<double2><<<g, 256, 0, st>>>((const double2 *)phi, pl.as<uint2>(), D);
    QS3_LAUNCHED();
    k_digitize<double2><<<dim3(B.nchunks, 1), XT, 0, st>>>(pl.as<uint2>(), D, 0, dgt.as<int2>(), get.as<int>(),
                                                           B.nchunks, B.d_secs.as<SecView>(), B.d_chunk0.as<int>(),
                                                           B.S);
    QS3_LAUNCHED();
    QS3_TRY(hphi_x_launch(B, phi, dgt.p, get.as<int>(), nullptr, psi, st, nullptr));
    QS3_CUDA(cudaStreamSynchronize(st));     // the scratch is released on return
    return QS3_OK;
}

}  // namespace qs3

extern "C" int qs3_gs_dots(qs3_basis_t b, qs3_dtype dtype, int32_t m, const void *V, uint64_t ldv, const void *w,
                           double *out, int32_t mode, void *stream) {
    clear_err();
    if (!b) return set_err(QS3_ERR_INVALID_ARG, "basis is NULL");
    if (m < 0) return set_err(QS3_ERR_INVALID_ARG, "m %d", m);
    if (m > 0 && (!V || !w || !out)) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    if (mode != 0 && mode != 1) return set_err(QS3_ERR_INVALID_ARG, "mode %d (need 0 or 1)", mode);
    Basis &B = b->B;
    if (m > 1 && ldv < B.total)
        return set_err(QS3_ERR_INVALID_ARG, "ldv %llu below the total dimension %llu", (unsigned long long)ldv,
                       (unsigned long long)B.total);
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == QS3_C128) return gs_dots_run<double2>(B, m, (const double2 *)V, ldv, (const double2 *)w, out, mode, st);
    if (dtype == QS3_F64) return gs_dots_run<double>(B, m, (const double *)V, ldv, (const double *)w, out, mode, st);
    return set_err(QS3_ERR_INVALID_ARG, "dtype %d (need F64 or C128)", (int)dtype);
}

// ------------------------------------------- dynamical structure factor
// Eq. (cfe): for every momentum q_n, psi_1 = S^-_q |gs> / |S^-_q gs| in the
// target sector n, n_iter Lanczos steps with full reorthogonalisation (Alg.
// 10 lines 3-11) batched over the n_q sectors, then the continued fraction
// evaluated on the omega grid by a device kernel.
namespace qs3 {

int cfrac_launch(int nq, int cap, const double *alpha, const double *beta, const int *msz, const double *norm2,
                 double e0, double h, double eta, const double *omega, int nw, double *out, cudaStream_t st);

int dsf_run(int op, Basis &S, int ss, const void *gs, double e0, Basis &Dd, int nq, const int *Q, int n_iter,
            double eta, double h, int nw, const double *omega, double *s_qw, double *alpha, double *beta,
            double *norm2, cudaStream_t st) {
    uint64_t nz = 0;
    QS3_TRY(count_nnz(Dd, &nz));
    HphiStats hs;
    Engine64<double2> E(Dd, st, &hs);
    QS3_TRY(E.init(n_iter + 1, 0));
    for (int n = 0; n < nq; ++n)
        QS3_TRY(sq_launch(op, S, ss, gs, Dd, n, Q + 3 * n, E.hin(0) + Dd.offs[n], st));
    QS3_TRY(E.normalise_start());
    std::vector<double2> n2(nq);
    QS3_CUDA(cudaMemcpyAsync(n2.data(), E.nrm.p, nq * sizeof(double2), cudaMemcpyDeviceToHost, st));
    QS3_CUDA(cudaStreamSynchronize(st));
    std::vector<double> nrm2(nq);
    for (int n = 0; n < nq; ++n) {
        nrm2[n] = Dd.dims[n] ? n2[n].x : 0.0;
        if (!(nrm2[n] > 0.0)) E.h_active[n] = 0;
        if (norm2) norm2[n] = nrm2[n];
    }
    QS3_TRY(E.push_active());
    for (int x = 0; x < n_iter && E.any_active(); ++x) QS3_TRY(E.step(x));
    QS3_TRY(E.check_err());
    std::vector<double> a, b;
    QS3_TRY(E.fetch(a, b));
    std::vector<int> msz(nq, 0);
    for (int n = 0; n < nq; ++n) {
        if (!(nrm2[n] > 0.0)) continue;
        int m = n_iter;
        for (int k = 0; k < n_iter - 1; ++k)
            if (b[(size_t)n * E.cap + k] == 0.0) { m = k + 1; break; }
        msz[n] = m;
        for (int x = 0; x < n_iter; ++x) {
            if (alpha) alpha[(size_t)n * n_iter + x] = x < m ? a[(size_t)n * E.cap + x] : 0.0;
            if (beta) beta[(size_t)n * n_iter + x] = x == 0 ? std::sqrt(nrm2[n])
                                                            : (x < m ? b[(size_t)n * E.cap + x - 1] : 0.0);
        }
    }
    if (s_qw && nw > 0) {
        DevBuf dm, dn, dw, dout;
        QS3_TRY(dm.upload(msz.data(), nq * sizeof(int)));
        QS3_TRY(dn.upload(nrm2.data(), nq * sizeof(double)));
        QS3_TRY(dw.upload(omega, nw * sizeof(double)));
        QS3_TRY(dout.alloc((size_t)nq * nw * sizeof(double)));
        // Zeeman shift of the resolvent: h times the change of N_down
        QS3_TRY(cfrac_launch(nq, E.cap, E.alpha.as<double>(), E.beta.as<double>(), dm.as<int>(), dn.as<double>(), e0,
                             h * (double)(Dd.nd - S.nd), eta, dw.as<double>(), nw, dout.as<double>(), st));
        QS3_CUDA(cudaMemcpyAsync(s_qw, dout.p, (size_t)nq * nw * sizeof(double), cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaStreamSynchronize(st));
    }
    return QS3_OK;
}

}  // namespace qs3

// ------------------------------------------------------ batched instances
// Many independent, uneven instances (different lattices, N_down, momenta):
// a pool of host workers, each driving its own non-blocking CUDA stream, takes
// the instances largest first and runs the batched-sector Lanczos of each; the
// GPU overlaps the instances' kernels.  An instance starts only when its
// Lanczos storage fits the memory budget next to the ones in flight (a single
// instance larger than the budget runs alone).
#include <condition_variable>
#include <mutex>
#include <thread>

namespace qs3 {

static size_t solve_mem_estimate(const Basis &B, const qs3_solve_opts &o) {
    const size_t ev = o.precision == QS3_F32 ? (B.has_k ? 8 : 4) : (B.has_k ? 16 : 8);
    const size_t ev64 = B.has_k ? 16 : 8;
    const size_t cap = (size_t)std::max(2, o.n_max) + 1;
    size_t m = cap * B.total * ev + 2 * B.total * ev64 + (size_t)std::max(B.nchunks, 1) * cap * 16;
    if (o.precision == QS3_F32) m += cap * B.total * ev64;   // the binary64 refinement
    m += 3 * B.total * ev64;                                 // w, H's input copy (and the double-float ring)
    if (o.precision != QS3_C128DF)       // the digit store and the exact-dot warp partials
        m += cap * B.total * ev64 + (size_t)std::max(B.nchunks, 1) * cap * XW * (24 + 4);
    if (B.has_k && o.precision == QS3_C128DF && !o.hphi_ieee) m += 2 * B.total * 16;   // double-float w and input
    return m;
}

static int batch_solve(int n, const qs3_basis_t *bases, const qs3_solve_opts &o, double *evals, void *const *evecs,
                       qs3_solve_info *infos, int maxc) {
    std::vector<size_t> off(n + 1, 0), mem(n);
    for (int i = 0; i < n; ++i) {
        if (!bases[i]) return set_err(QS3_ERR_INVALID_ARG, "basis %d is NULL", i);
        off[i + 1] = off[i] + bases[i]->B.S;
        mem[i] = solve_mem_estimate(bases[i]->B, o);
        uint64_t nz;
        QS3_TRY(count_nnz(bases[i]->B, &nz));        // on the calling thread, before the workers start
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mem[a] > mem[b]; });
    int dev = 0;
    QS3_CUDA(cudaGetDevice(&dev));
    size_t freeb = 0, totb = 0;
    QS3_CUDA(cudaMemGetInfo(&freeb, &totb));
    const size_t budget = (size_t)(0.85 * (double)freeb);
    std::mutex mu;
    std::condition_variable cv;
    size_t inflight = 0;
    int nrun = 0, next = 0, first_err = QS3_OK;
    std::string err_text;
    std::vector<qs3_solve_info> inf(n);
    std::vector<int> status(n, QS3_OK);
    auto worker = [&]() {
        cudaSetDevice(dev);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            if (first_err == QS3_OK) { first_err = QS3_ERR_CUDA; err_text = "stream creation failed"; }
            return;
        }
        for (;;) {
            int i;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (next >= n || first_err != QS3_OK) break;
                i = order[next];
                cv.wait(lk, [&] { return first_err != QS3_OK || nrun == 0 || inflight + mem[i] <= budget; });
                if (first_err != QS3_OK) break;
                if (order[next] != i) continue;      // another worker took it meanwhile
                ++next;
                inflight += mem[i];
                ++nrun;
            }
            Basis &B = bases[i]->B;
            qs3_solve_info info{};
            int s = B.has_k ? lanczos_entry<float2, double2>(B, o, evals + off[i], evecs ? evecs[i] : nullptr, &info, st)
                            : lanczos_entry<float, double>(B, o, evals + off[i], evecs ? evecs[i] : nullptr, &info, st);
            {
                std::lock_guard<std::mutex> lk(mu);
                inf[i] = info;
                status[i] = s;
                inflight -= mem[i];
                --nrun;
                if (s != QS3_OK && s != QS3_ERR_NOT_CONVERGED && first_err == QS3_OK) {
                    first_err = s;
                    err_text = last_err();
                }
            }
            cv.notify_all();
        }
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    };
    const int nw = std::max(1, std::min(n, maxc > 0 ? maxc : 16));
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
    for (auto &t : pool) t.join();
    if (infos)
        for (int i = 0; i < n; ++i) infos[i] = inf[i];
    if (first_err != QS3_OK) return set_err(first_err, "batch: %s", err_text.c_str());
    for (int i = 0; i < n; ++i)
        if (status[i] == QS3_ERR_NOT_CONVERGED) return set_err(QS3_ERR_NOT_CONVERGED, "batch: instance %d did not converge", i);
    return QS3_OK;
}

}  // namespace qs3

extern "C" int qs3_batch_solve(int32_t n, const qs3_basis_t *bases, const qs3_solve_opts *o, double *evals,
                               void *const *evecs, qs3_solve_info *infos, int32_t max_concurrent) {
    qs3::clear_err();
    if (n < 0 || (n > 0 && (!bases || !evals))) return qs3::set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    QS3_TRY(qs3::check_opts(o));
    if (n == 0) return QS3_OK;
    return qs3::batch_solve(n, bases, *o, evals, evecs, infos, max_concurrent);
}
