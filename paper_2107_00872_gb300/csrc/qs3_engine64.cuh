// qs3_engine64.cuh -- the IEEE binary64 Lanczos engine of fp64 solves
// (included by qs3_solver.cu after the kernels it reuses).
//
// Alg. 10 in the paper's arithmetic, complex double (k-sectors) or double
// (U(1)-only bases): every Lanczos vector, every product H psi_x and every
// Gram-Schmidt operand is an IEEE binary64 value.
//
// Layout.  The Krylov basis is kept as binary64 values split into their high
// and low 32-bit words, stored in two planes per vector (word-planar): slot j
// holds D high words (complex: (re.hi, im.hi) pairs) and then D low words.
// A value is reassembled bit for bit from its two words.  Beside it a digit
// store holds each vector's fixed-point image (below).  The product H psi_x
// reads an interleaved copy of psi_x (hin) written together with slot x.
//
// One step (Alg. 10 lines 5-11, full reorthogonalisation):
//   w = H psi_x;  alpha_x = Re psi_x^H w;  w -= beta_{x-1} psi_{x-1} +
//   alpha_x psi_x (the recurrence, real scalars);  one classical
//   Gram-Schmidt pass: g_j = psi_j^H w for j = 0..x, w -= sum_j g_j psi_j
//   (it also removes what the recurrence left along psi_x, psi_{x-1});
//   beta_x = |w|;  psi_{x+1} = w / beta_x.  The first step after a thick
//   restart runs a full first pass with complex coefficients instead of the
//   recurrence.  The Gram-Schmidt kernels read the digit store either with
//   register staging (k_dotx, k_upd64) or through shared-memory rings filled
//   by bulk asynchronous copies (k_dotb, k_updb), as the autotuner chooses.
// Updates are binary64 FMA chains per thread.  Two exceptions, both bounded
// below binary64's own rounding:
//  - the dot products are exact sums on fixed-point images of the operands
//    (k_dotx, below; the stored vectors' images are kept in a digit store);
//  - the Gram-Schmidt update whose coefficients are all tiny: when
//    sum_j |g_j| <= 2^-40 |w| (the normal case: w is already orthogonal to
//    the basis to O(eps)), the correction u = sum_j g_j psi_j is summed in
//    fp32 from the top digits of the digit store (each value known to 2^-21
//    of its warp group's largest magnitude, so |delta psi_j| <= 2^-17.5 in
//    norm), and the fp32 sums of m <= 2^8 terms add relative 2^-16:
//    |error of u| <= (2^-17.5 + 2^-16) 2^-40 |w| < 2^-55.5 |w|, below half an
//    ulp of binary64 applied to |w| (for m > 2^8 the limit 2^-40 shrinks by
//    2^8 / m); w - u is then formed in binary64.
// The solve option strict64 keeps the dots and that update on binary64 FMAs.
#pragma once

#include "qs3_fixed.cuh"

namespace qs3 {

template <typename VT> struct PlS { using T = uint32_t; };     // real: one word per plane
template <> struct PlS<double2> { using T = uint2; };          // complex: (re, im) words per plane

__device__ __forceinline__ double2 pl_ld(const uint2 *slot, uint64_t D, uint64_t r) {
    const uint2 h = slot[r], l = slot[D + r];
    return make_double2(__hiloint2double((int)h.x, (int)l.x), __hiloint2double((int)h.y, (int)l.y));
}
__device__ __forceinline__ double2 pl_ld(const uint32_t *slot, uint64_t D, uint64_t r) {
    return make_double2(__hiloint2double((int)slot[r], (int)slot[D + r]), 0.0);
}
__device__ __forceinline__ void pl_st(uint2 *slot, uint64_t D, uint64_t r, double2 v) {
    slot[r] = make_uint2((unsigned)__double2hiint(v.x), (unsigned)__double2hiint(v.y));
    slot[D + r] = make_uint2((unsigned)__double2loint(v.x), (unsigned)__double2loint(v.y));
}
__device__ __forceinline__ void pl_st(uint32_t *slot, uint64_t D, uint64_t r, double2 v) {
    slot[r] = (unsigned)__double2hiint(v.x);
    slot[D + r] = (unsigned)__double2loint(v.x);
}

// part[c * m + j] = conj(V_{j0+j}) . w over chunk c (binary64 FMAs); V the
// word-planar store (slots of 2D words-per-element units), w interleaved.
// Vectors go in groups of 8 (partial sums of a group meet in shared memory,
// warp q reduces vector q); NV vectors per pass have their loads in flight
// together.  Graph mode (dx): the range of graph_range.
template <typename VT, int NV>
__global__ void __launch_bounds__(NTHREADS, NV == 1 ? 3 : NV == 2 ? 2 : 1)
    k_dot64(const typename PlS<VT>::T *__restrict__ V, uint64_t D, int j0, int m, const VT *__restrict__ w,
            const SecView *__restrict__ secs, const int *__restrict__ chunk0, int S, const int *__restrict__ active,
            double2 *__restrict__ part, const int *__restrict__ dx = nullptr, int ring = 0) {
    using T = typename PlS<VT>::T;
    constexpr bool CX = IsC<VT>::v;
    __shared__ double2 red[GDF][NTHREADS];
    graph_range(dx, ring, j0, m);
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (ci.n - (int)threadIdx.x + NTHREADS - 1) / NTHREADS;     // rows of this thread
    const uint64_t r0 = ci.base + threadIdx.x;
    double2 wv[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) wv[k] = k < nk ? ld2(w + r0 + (uint64_t)k * NTHREADS) : make_double2(0.0, 0.0);
    for (int jb = 0; jb < m; jb += GDF) {
        const int nj = min(GDF, m - jb);
        for (int jj = 0; jj < nj; jj += NV) {
            double2 a[NV][RPT];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int jv = jj + v < nj ? jj + v : nj - 1;      // past the group: a repeat, discarded
                const T *slot = V + (uint64_t)(j0 + jb + jv) * 2 * D;
#pragma unroll
                for (int k = 0; k < RPT; ++k)
                    a[v][k] = k < nk ? pl_ld(slot, D, r0 + (uint64_t)k * NTHREADS) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double2 acc = make_double2(0.0, 0.0);
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    const double2 x = a[v][k], b = wv[k];
                    // conj(x) b = (x.r b.r + x.i b.i) + i (x.r b.i - x.i b.r)
                    acc.x = fma(x.x, b.x, acc.x);
                    if (CX) {
                        acc.x = fma(x.y, b.y, acc.x);
                        acc.y = fma(x.x, b.y, acc.y);
                        acc.y = fma(-x.y, b.x, acc.y);
                    }
                }
                if (jj + v < nj) red[jj + v][threadIdx.x] = acc;
            }
        }
        __syncthreads();
        if (warp < nj) {
            double2 t = make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < NTHREADS / 32; ++q) {
                const double2 v = red[warp][lane + 32 * q];
                t.x += v.x;
                t.y += v.y;
            }
            t = warp_sum2(t);
            if (lane == 0) part[(uint64_t)blockIdx.x * m + jb + warp] = t;
        }
        __syncthreads();
    }
}

// ------------------------------------------------ exact fixed-point dots
// The fp64 pipe of this GPU retires one FMA per ~70 fp32 FMAs, so a complex
// binary64 dot (4 DFMA per 16 bytes) cannot pass ~2.1 TB/s, a third of HBM.
// k_dotx forms the same dot products on the integer units, exactly:
//  - every operand is rounded once (to nearest) onto a fixed-point grid set
//    by the largest exponent among its warp's rows: for biased exponent em,
//    v -> P = round(v 2^(1075 - em)), |P| <= 2^53, an error of at most
//    2^-53 of the warp's largest magnitude (binary64 rounds its largest
//    element by as much);
//  - P is split into balanced base-2^26 digits P = P1 2^26 + P0 (|P0| <=
//    2^25, |P1| <= 2^27 + 1); the digit products P1 W1 (weight 2^52) and
//    P1 W0 + P0 W1 (weight 2^26) are summed exactly in 64-bit integers
//    (mad.wide.s32); P0 W0 (at most 2^50, random in sign: a quarter of the
//    grid error) is left out;
//  - each thread folds its middle sum into its top sum (rounded to nearest
//    at weight 2^52), the warp adds its 32 threads' sums exactly
//    (redux.sync on 26-bit limbs) and writes them with its grid exponent;
//  - k_reducex aligns the warp sums of every chunk of a sector to the
//    coarsest grid among them (rounded to nearest), adds them exactly in
//    128-bit integers and rounds the sector's dot to binary64 once.
// Neither kernel issues an fp64 instruction on the normal path.
// Bounds: a thread's folded sum (8 top-digit products of <= 2^54.1 and 16
// middle ones of <= 2^52.1 for complex data) stays below 2^57.2, a warp's
// below 2^62.2.
// the sum over the warp of t, |t| < 2^58: three limbs of at most 26 bits,
// whose 32-lane sums fit in int32, each summed by one redux.sync
__device__ __forceinline__ long long warp_sum_ll(long long t) {
    const int l0 = (int)(t & 0x3ffffffll);
    const int l1 = (int)((t >> 26) & 0x3ffffffll);
    const int l2 = (int)(t >> 52);
    const long long s0 = __reduce_add_sync(0xffffffffu, l0);
    const long long s1 = __reduce_add_sync(0xffffffffu, l1);
    const long long s2 = __reduce_add_sync(0xffffffffu, l2);
    return s0 + s1 * (1ll << 26) + s2 * (1ll << 52);
}
// the sum over the warp of a 128-bit value (exact, all lanes)
__device__ __forceinline__ __int128 warp_sum_i128(__int128 v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
        const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, o), ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        v += (__int128)(((unsigned __int128)ohi << 64) | olo);
    }
    return v;
}
__device__ __forceinline__ void words(uint2 h, uint2 l, uint32_t (&hw)[2], uint32_t (&lw)[2]) {
    hw[0] = h.x; hw[1] = h.y; lw[0] = l.x; lw[1] = l.y;
}
__device__ __forceinline__ void words(uint32_t h, uint32_t l, uint32_t (&hw)[2], uint32_t (&lw)[2]) {
    hw[0] = h; hw[1] = 0u; lw[0] = l; lw[1] = 0u;
}

// The digit store.  Every stored vector also exists as its fixed-point
// image: per row the balanced digits (P1, P0) of each component, in two
// planes per slot (D P1 words: (re, im) pairs for complex rows, then D P0
// words), and per chunk and warp group (the 128 rows base + 32 q + lane +
// 512 k of a chunk) the grid exponent em.  It is derived from the binary64
// store by the kernels that write it (k_scale64, k_digitize) and read by the
// dot products (both planes) and the fp32 Gram-Schmidt correction (P1 only).
template <typename VT> struct DigT { using T = int; };
template <> struct DigT<double2> { using T = int2; };

__device__ __forceinline__ void dig_st(int2 *slot, uint64_t D, uint64_t r, const int (&d1)[2], const int (&d0)[2]) {
    slot[r] = make_int2(d1[0], d1[1]);
    slot[D + r] = make_int2(d0[0], d0[1]);
}
__device__ __forceinline__ void dig_st(int *slot, uint64_t D, uint64_t r, const int (&d1)[2], const int (&d0)[2]) {
    slot[r] = d1[0];
    slot[D + r] = d0[0];
}
__device__ __forceinline__ void dig_ld(const int2 *slot, uint64_t D, uint64_t r, int (&d1)[2], int (&d0)[2]) {
    const int2 h = slot[r], l = slot[D + r];
    d1[0] = h.x; d1[1] = h.y; d0[0] = l.x; d0[1] = l.y;
}
__device__ __forceinline__ void dig_ld(const int *slot, uint64_t D, uint64_t r, int (&d1)[2], int (&d0)[2]) {
    d1[0] = slot[r]; d1[1] = 0; d0[0] = slot[D + r]; d0[1] = 0;
}
// the top digit P1 (|P1| <= 2^27) as the float P1 / 32 rounded down to an
// integer (|.| <= 2^22, exact: 1.5 2^23 + x has unit spacing)
__device__ __forceinline__ float p1_f(int p1) { return __int_as_float(0x4B400000 + (p1 >> 5)) - 12582912.0f; }
__device__ __forceinline__ float2 p1_f2(int2 p) { return make_float2(p1_f(p.x), p1_f(p.y)); }
__device__ __forceinline__ float2 p1_f2(int p) { return make_float2(p1_f(p), 0.f); }

// the XR binary64 values (hi, lo words per component) of one thread of a
// warp group on the group's grid: the warp's largest biased exponent em
// (at least 54) and the digits of every value
template <int NC>
__device__ __forceinline__ int fx_group(const uint32_t (&hw)[XR][2], const uint32_t (&lw)[XR][2], int (&d1)[XR][2],
                                        int (&d0)[XR][2]) {
    int em = 54;
#pragma unroll
    for (int k = 0; k < XR; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) em = max(em, fx_exp(hw[k][c]));
    em = (int)__reduce_max_sync(0xffffffffu, (unsigned)em);
#pragma unroll
    for (int k = 0; k < XR; ++k)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c < NC) fx_digits(hw[k][c], lw[k][c], em, d1[k][c], d0[k][c]);
            else d1[k][c] = d0[k][c] = 0;
        }
    return em;
}

// w's digits as the dot products use them: per row the top and low digits
// (w1, w0) of each component and, for complex rows, those of w.r + w.i (e)
// and w.i - w.r (f), each the sum of the components' digits
struct WDig {
    int w1[XR][2], w0[XR][2], e1[XR], e0[XR], f1[XR], f0[XR];
    __device__ __forceinline__ void pairs() {
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            e1[k] = w1[k][0] + w1[k][1];
            e0[k] = w0[k][0] + w0[k][1];
            f1[k] = w1[k][1] - w1[k][0];
            f0[k] = w0[k][1] - w0[k][0];
        }
    }
};

// One thread's share of conj(a) . w over its XR rows: the sum of the top
// digit products (weight 2^52) plus the sum of the middle ones (weight 2^26)
// rounded to nearest at 2^52; the low x low products are dropped.  Complex
// rows take three products per digit pair instead of four, from
//   re = w.r s + a.i (w.r + w.i),  im = w.r s + a.r (w.i - w.r),  s = a.r - a.i:
// the digits of s, w.r + w.i and w.i - w.r are sums of the operands' digits,
// so the top, middle and dropped sums are the same integers as those of
// (a.r w.r + a.i w.i) + i (a.r w.i - a.i w.r) taken product by product.
// Bounds: digits of s, e, f below 2^28 (top) and 2^26 (low), so every
// product and every partial sum here stays far inside 64 bits.
template <bool CX>
__device__ __forceinline__ void fx_thread_dot(const int (&a1)[XR][2], const int (&a0)[XR][2], const WDig &d,
                                              long long &tr, long long &ti) {
    if constexpr (CX) {
        long long hk = 0, mk = 0, h3 = 0, m3 = 0, h2 = 0, m2 = 0;
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            const int s1 = a1[k][0] - a1[k][1], s0 = a0[k][0] - a0[k][1];
            hk = mad_w(d.w1[k][0], s1, hk);
            mk = mad_w(d.w1[k][0], s0, mk);
            mk = mad_w(d.w0[k][0], s1, mk);
            h3 = mad_w(a1[k][1], d.e1[k], h3);
            m3 = mad_w(a1[k][1], d.e0[k], m3);
            m3 = mad_w(a0[k][1], d.e1[k], m3);
            h2 = mad_w(a1[k][0], d.f1[k], h2);
            m2 = mad_w(a1[k][0], d.f0[k], m2);
            m2 = mad_w(a0[k][0], d.f1[k], m2);
        }
        tr = (hk + h3) + ((mk + m3 + (1ll << 25)) >> 26);
        ti = (hk + h2) + ((mk + m2 + (1ll << 25)) >> 26);
    } else {
        long long h = 0, m1 = 0, m0 = 0;
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            h = mad_w(a1[k][0], d.w1[k][0], h);
            m1 = mad_w(a1[k][0], d.w0[k][0], m1);
            m0 = mad_w(a0[k][0], d.w1[k][0], m0);
        }
        tr = h + ((m1 + m0 + (1ll << 25)) >> 26);
        ti = 0;
    }
}

// digit store slots j0 .. j0 + gridDim.y - 1 from the binary64 store (one
// block of XT threads per chunk)
template <typename VT>
__global__ void __launch_bounds__(XT)
    k_digitize(const typename PlS<VT>::T *__restrict__ V, uint64_t D, int j0, typename DigT<VT>::T *__restrict__ dg,
               int *__restrict__ ge, int nchunks, const SecView *__restrict__ secs, const int *__restrict__ chunk0,
               int S) {
    using T = typename PlS<VT>::T;
    constexpr int NC = IsC<VT>::v ? 2 : 1;
    const int j = j0 + blockIdx.y;
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *slot = V + (uint64_t)j * 2 * D;
    uint32_t hw[XR][2], lw[XR][2];
#pragma unroll
    for (int k = 0; k < XR; ++k) {
        const int r = threadIdx.x + k * XT;
        const T h = r < ci.n ? slot[ci.base + r] : T{};
        const T l = r < ci.n ? slot[D + ci.base + r] : T{};
        words(h, l, hw[k], lw[k]);
    }
    int d1[XR][2], d0[XR][2];
    const int em = fx_group<NC>(hw, lw, d1, d0);
    typename DigT<VT>::T *out = dg + (uint64_t)j * 2 * D;
#pragma unroll
    for (int k = 0; k < XR; ++k) {
        const int r = threadIdx.x + k * XT;
        if (r < ci.n) dig_st(out, D, ci.base + r, d1[k], d0[k]);
    }
    if (lane == 0) ge[((uint64_t)j * nchunks + blockIdx.x) * XW + warp] = em;
}

// The exact dot products conj(V_{j0+j}) . w over chunk c, as warp partials:
// part[((c m + j) XW + q) 3 + {0, 1, 2}] = the re and im sums of warp q (in
// units of 2^(k - 2098)) and k = em + ew, the sum of its two grid exponents.
// The stored vectors are read from the digit store (dg, ge), w (interleaved
// binary64) is put on its warps' grids here.  NV vectors per pass have their
// loads in flight together.  Graph mode (dx): the range of graph_range.
template <typename VT, int NV>
__global__ void __launch_bounds__(XT, 1)
    k_dotx(const typename DigT<VT>::T *__restrict__ dg, const int *__restrict__ ge, int nchunks, uint64_t D, int j0,
           int m, const VT *__restrict__ w, const SecView *__restrict__ secs, const int *__restrict__ chunk0, int S,
           const int *__restrict__ active, long long *__restrict__ part, const int *__restrict__ dx = nullptr,
           int ring = 0) {
    using G = typename DigT<VT>::T;
    constexpr bool CX = IsC<VT>::v;
    constexpr int NC = CX ? 2 : 1;
    graph_range(dx, ring, j0, m);
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (ci.n - (int)threadIdx.x + XT - 1) / XT;          // rows of this thread
    const uint64_t r0 = ci.base + threadIdx.x;
    // w on its warp's grid: digits per row and component
    WDig wd;
    int ew;
    {
        uint32_t hw[XR][2], lw[XR][2];
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            const double2 v = k < nk ? ld2(w + r0 + (uint64_t)k * XT) : make_double2(0.0, 0.0);
            hw[k][0] = (uint32_t)__double2hiint(v.x);
            lw[k][0] = (uint32_t)__double2loint(v.x);
            hw[k][1] = (uint32_t)__double2hiint(v.y);
            lw[k][1] = (uint32_t)__double2loint(v.y);
        }
        ew = fx_group<NC>(hw, lw, wd.w1, wd.w0);
        wd.pairs();
    }
    // NV stored vectors per stage, two stages: the loads of the next stage
    // are in flight while the current one is multiplied
    struct Stage {
        int a1[NV][XR][2], a0[NV][XR][2], em[NV];
    };
    auto load = [&](Stage &b, int jj) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int jv = j0 + (jj + v < m ? jj + v : m - 1);      // past the end: a repeat, discarded
            const G *slot = dg + (uint64_t)jv * 2 * D;
            b.em[v] = ge[((uint64_t)jv * nchunks + blockIdx.x) * XW + warp];
#pragma unroll
            for (int k = 0; k < XR; ++k) {
                if (k < nk) {
                    dig_ld(slot, D, r0 + (uint64_t)k * XT, b.a1[v][k], b.a0[v][k]);
                } else {
                    b.a1[v][k][0] = b.a0[v][k][0] = b.a1[v][k][1] = b.a0[v][k][1] = 0;
                }
            }
        }
    };
    auto consume = [&](const Stage &b, int jj) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            long long tr, ti;
            fx_thread_dot<CX>(b.a1[v], b.a0[v], wd, tr, ti);
            const long long sr = warp_sum_ll(tr);
            const long long si = CX ? warp_sum_ll(ti) : 0ll;
            if (lane == 0 && jj + v < m) {
                long long *o = part + (((uint64_t)blockIdx.x * m + jj + v) * XW + warp) * 3;
                o[0] = sr;
                o[1] = si;
                o[2] = b.em[v] + ew;
            }
        }
    };
    Stage s0, s1;
    if (m > 0) load(s0, 0);
#pragma unroll 1
    for (int jj = 0; jj < m; jj += 2 * NV) {
        if (jj + NV < m) load(s1, jj + NV);
        consume(s0, jj);
        if (jj + NV >= m) break;
        if (jj + 2 * NV < m) load(s0, jj + 2 * NV);
        consume(s1, jj + NV);
    }
}

// The same dot products with the stored vectors' digits brought in by TMA
// bulk copies (k_dotb).  A producer warp (warp XW, one elected lane) copies,
// per stored vector, the chunk's slices of both digit planes and its XW group
// exponents into stage jj % NS of a ring in shared memory (complete_tx on the
// stage's "full" mbarrier); each of the XW consumer warps multiplies the
// stage and arrives on its "empty" mbarrier, which the producer waits for
// before refilling the stage.  A slice starts at the 16-byte boundary at or
// below the chunk's first element (off elements earlier, off computed per
// plane) and its size is rounded up to 16 bytes: the store must have 16
// readable bytes past its end.  Every wait is bounded by the global timer
// (MB_NS nanoseconds): a wait that runs out sets *err, the warp leaves its
// loop, and the producer waits (bounded) for the copies it has in flight
// before it exits, so that no copy lands in a finished block's memory.
// starve != 0 (the test injection of a lost copy): the producer issues no
// copies, so the consumers' first waits run out.
constexpr unsigned long long MB_NS = 1000000000ull;     // 1 s

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// wait for the completion of the phase with the given parity, at most MB_NS
// nanoseconds; false when the wait ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try(b, parity))
        if (gtimer() - t0 > MB_NS) return false;
    return true;
}
// orders this thread's view of earlier generic-proxy accesses to shared
// memory (the consumers' reads of a stage, observed through its empty
// barrier) before the bulk copies it issues next (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// one ring stage: two digit slices (a chunk plus up to 16 bytes before it,
// rounded up to 16 bytes), then the chunk's XW group exponents
template <typename VT> constexpr unsigned dotb_slice() {
    return (unsigned)((BROWS * sizeof(typename DigT<VT>::T) + 16 + 15) / 16 * 16);
}
template <typename VT> constexpr unsigned dotb_stage() { return 2 * dotb_slice<VT>() + XW * 4; }
template <typename VT, int NS> constexpr unsigned dotb_smem() { return NS * dotb_stage<VT>(); }

template <typename VT, int NS>
__global__ void __launch_bounds__(XT + 32, 1)
    k_dotb(const typename DigT<VT>::T *__restrict__ dg, const int *__restrict__ ge, int nchunks, uint64_t D, int j0,
           int m, const VT *__restrict__ w, const SecView *__restrict__ secs, const int *__restrict__ chunk0, int S,
           const int *__restrict__ active, long long *__restrict__ part, int *__restrict__ err, int starve,
           const int *__restrict__ dx = nullptr, int ring = 0) {
    using G = typename DigT<VT>::T;
    constexpr bool CX = IsC<VT>::v;
    constexpr int NC = CX ? 2 : 1;
    constexpr unsigned SL = dotb_slice<VT>(), SB = dotb_stage<VT>();
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    graph_range(dx, ring, j0, m);
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int t = 0; t < NS; ++t) {
            mbar_init(&full[t], 1);
            mbar_init(&empty[t], XW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the chunk's first element in plane pl of stored vector jj, and its byte
    // offset above the 16-byte boundary: that of vector 0 plus jj times the
    // slot size (2 D elements) modulo 16
    auto plane = [&](int jj, int pl) { return dg + ((uint64_t)(j0 + jj) * 2 + pl) * D + ci.base; };
    auto offb = [&](const G *p) { return (unsigned)((uintptr_t)p & 15u); };
    const unsigned ob1 = offb(plane(0, 0)), ob0 = offb(plane(0, 1));
    const unsigned osl = (unsigned)(2 * D * sizeof(G)) & 15u;
    auto offj = [&](unsigned ob, int jj) { return (ob + (unsigned)jj * osl) & 15u; };
    if (warp == XW) {
        // producer
        if (lane == 0) {
            const unsigned nb = (unsigned)ci.n * (unsigned)sizeof(G);
            int issued = 0;
            bool ok = true;
            for (; issued < m && !starve; ++issued) {
                const int t = issued % NS;
                if (issued >= NS) {
                    if (!mbar_wait(&empty[t], (unsigned)(issued / NS - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();
                }
                unsigned char *sp = dsm + (size_t)t * SB;
                const G *p1 = plane(issued, 0), *p0 = plane(issued, 1);
                const unsigned o1 = offb(p1), o0 = offb(p0);
                const unsigned b1 = (o1 + nb + 15u) & ~15u, b0 = (o0 + nb + 15u) & ~15u;
                mbar_expect_tx(&full[t], b1 + b0 + XW * 4);
                bulk_g2s(sp, (const unsigned char *)p1 - o1, b1, &full[t]);
                bulk_g2s(sp + SL, (const unsigned char *)p0 - o0, b0, &full[t]);
                bulk_g2s(sp + 2 * SL, ge + ((uint64_t)(j0 + issued) * nchunks + blockIdx.x) * XW, XW * 4, &full[t]);
            }
            if (!ok) atomicExch(err, 1);
            // the copies in flight land before the block ends
            for (int jj = issued - NS > 0 ? issued - NS : 0; jj < issued; ++jj)
                mbar_wait(&full[jj % NS], (unsigned)(jj / NS) & 1u);
        }
        return;
    }
    const int nk = (ci.n - (int)threadIdx.x + XT - 1) / XT;          // rows of this thread
    const uint64_t r0 = ci.base + threadIdx.x;
    // w on its warp's grid
    WDig wd;
    int ew;
    {
        uint32_t hw[XR][2], lw[XR][2];
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            const double2 v = k < nk ? ld2(w + r0 + (uint64_t)k * XT) : make_double2(0.0, 0.0);
            hw[k][0] = (uint32_t)__double2hiint(v.x);
            lw[k][0] = (uint32_t)__double2loint(v.x);
            hw[k][1] = (uint32_t)__double2hiint(v.y);
            lw[k][1] = (uint32_t)__double2loint(v.y);
        }
        ew = fx_group<NC>(hw, lw, wd.w1, wd.w0);
        wd.pairs();
    }
    // the thread's folded sums of one stored vector (fx_thread_dot)
    auto tsum = [&](const unsigned char *sp, int jj, long long &tr, long long &ti) {
        const G *p1 = (const G *)(sp + offj(ob1, jj));
        const G *p0 = (const G *)(sp + SL + offj(ob0, jj));
        int a1[XR][2], a0[XR][2];
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            a1[k][0] = a1[k][1] = a0[k][0] = a0[k][1] = 0;
            if (k < nk) {
                const G q1 = p1[threadIdx.x + k * XT], q0 = p0[threadIdx.x + k * XT];
                if constexpr (CX) {
                    a1[k][0] = q1.x; a1[k][1] = q1.y; a0[k][0] = q0.x; a0[k][1] = q0.y;
                } else {
                    a1[k][0] = q1; a0[k][0] = q0;
                }
            }
        }
        fx_thread_dot<CX>(a1, a0, wd, tr, ti);
    };
    // two stored vectors per pass (their chains interleave); lane 0 waits
    // for the stages, then every lane observes the completed phases itself
#pragma unroll 1
    for (int jj = 0; jj < m; jj += 2) {
        const bool two = jj + 1 < m;
        const int t0 = jj % NS, t1 = (jj + 1) % NS;
        const unsigned q0 = (unsigned)(jj / NS) & 1u, q1 = (unsigned)((jj + 1) / NS) & 1u;
        bool ok = true;
        if (lane == 0) {
            ok = mbar_wait(&full[t0], q0);
            if (ok && two) ok = mbar_wait(&full[t1], q1);
        }
        if (!__shfl_sync(0xffffffffu, (int)ok, 0)) {
            // a wait ran out: record it and leave zero partials for the
            // vectors not multiplied, so that what follows stays finite
            if (lane == 0) {
                atomicExch(err, 1);
                for (int j = jj; j < m; ++j) {
                    long long *o = part + (((uint64_t)blockIdx.x * m + j) * XW + warp) * 3;
                    o[0] = 0;
                    o[1] = 0;
                    o[2] = ew + 54;
                }
            }
            break;
        }
        mbar_try(&full[t0], q0);
        if (two) mbar_try(&full[t1], q1);
        const unsigned char *s0 = dsm + (size_t)t0 * SB, *s1 = dsm + (size_t)t1 * SB;
        long long tr0, ti0, tr1 = 0, ti1 = 0;
        const int em0 = ((const int *)(s0 + 2 * SL))[warp];
        const int em1 = two ? ((const int *)(s1 + 2 * SL))[warp] : 0;
        tsum(s0, jj, tr0, ti0);
        if (two) tsum(s1, jj + 1, tr1, ti1);
        // both stages are read: release them to the producer
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&empty[t0]);
            if (two) mbar_arrive(&empty[t1]);
        }
        const long long sr0 = warp_sum_ll(tr0), sr1 = warp_sum_ll(tr1);
        const long long si0 = CX ? warp_sum_ll(ti0) : 0ll, si1 = CX ? warp_sum_ll(ti1) : 0ll;
        if (lane == 0) {
            long long *o = part + (((uint64_t)blockIdx.x * m + jj) * XW + warp) * 3;
            o[0] = sr0;
            o[1] = si0;
            o[2] = em0 + ew;
            if (two) {
                o += XW * 3;
                o[0] = sr1;
                o[1] = si1;
                o[2] = em1 + ew;
            }
        }
    }
}

// The sector sums of the k_dotx partials, exactly, in two levels so that a
// sector of many chunks is reduced by many warps: k_reducex1 takes slices of
// RSL (chunk, warp) partials of one sector, aligns them to the coarsest grid
// in the slice (rounded to nearest) and sums them in 128 bits; k_reducex2
// aligns the slice sums of a sector the same way, sums them and rounds to
// binary64 once.  A warp partial s at exponent sum k is worth s 2^(k - 2098).
constexpr int RSL = 4096;

// first slice of every sector (S + 1 entries)
static inline std::vector<int> reduce_slices(const Basis &B) {
    std::vector<int> s0(B.S + 1, 0);
    for (int s = 0; s < B.S; ++s) {
        const int parts = (B.chunk0[s + 1] - B.chunk0[s]) * XW;
        s0[s + 1] = s0[s] + (parts + RSL - 1) / RSL;
    }
    return s0;
}
// every sector has exactly one slice (the first level then finishes)
static inline bool one_slice(const std::vector<int> &s0) {
    for (size_t s = 0; s + 1 < s0.size(); ++s)
        if (s0[s + 1] - s0[s] != 1) return false;
    return s0.size() > 1;
}

__device__ __forceinline__ __int128 align_round(__int128 v, int d) {
    if (d <= 0) return v;
    if (d > 120) return 0;
    return (v + ((__int128)1 << (d - 1))) >> d;
}

// out1[(sl m + j) 5 + {0..4}] = re (lo, hi words), im (lo, hi), K of slice sl
// and coefficient j; one warp per coefficient (graph mode: graph_range)
__global__ void k_reducex1(const long long *__restrict__ part, int m, const int *__restrict__ chunk0,
                           const int *__restrict__ slice0, int S, const int *__restrict__ active,
                           long long *__restrict__ out1, const int *__restrict__ dx, int ring,
                           double2 *__restrict__ out = nullptr, int ldo = 0, int cx = 1) {
    if (dx) {
        int j0 = 0;
        graph_range(dx, ring, j0, m);
        if (out) out += j0;               // the one-level form only
    }
    const int sl = blockIdx.x;
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (slice0[mid] <= sl) lo = mid; else hi = mid - 1;
    }
    const int s = lo;
    if (active && !active[s]) return;
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= m) return;
    const int p0 = chunk0[s] * XW + (sl - slice0[s]) * RSL, p1 = min(p0 + RSL, chunk0[s + 1] * XW);
    int K = -1;
    for (int p = p0 + lane; p < p1; p += 32) {
        const long long *q = part + (((uint64_t)(p / XW) * m + j) * XW + p % XW) * 3;
        K = max(K, (int)q[2]);
    }
    K = __reduce_max_sync(0xffffffffu, K);
    __int128 ar = 0, ai = 0;
    for (int p = p0 + lane; p < p1; p += 32) {
        const long long *q = part + (((uint64_t)(p / XW) * m + j) * XW + p % XW) * 3;
        const int d = K - (int)q[2];
        ar += align_round(q[0], d);
        ai += align_round(q[1], d);
    }
    ar = warp_sum_i128(ar);
    ai = warp_sum_i128(ai);
    if (out) {
        // one slice per sector: the slice sum is the sector's dot
        if (lane == 0)
            out[(uint64_t)s * ldo + j] = make_double2(i128_ldexp(ar, K - 2098), cx ? i128_ldexp(ai, K - 2098) : 0.0);
        return;
    }
    if (lane == 0) {
        long long *o = out1 + ((uint64_t)sl * m + j) * 5;
        o[0] = (long long)(unsigned long long)ar;
        o[1] = (long long)(ar >> 64);
        o[2] = (long long)(unsigned long long)ai;
        o[3] = (long long)(ai >> 64);
        o[4] = K;
    }
}

// out[s * ldo + j] from the slice sums of sector s (graph mode: the range of
// graph_range, written from out + j0); one warp per coefficient
__global__ void k_reducex2(const long long *__restrict__ out1, int m, const int *__restrict__ slice0,
                           const int *__restrict__ active, double2 *__restrict__ out, int ldo,
                           const int *__restrict__ dx, int ring, int cx) {
    const int s = blockIdx.y;
    if (dx) {
        int j0 = 0;
        graph_range(dx, ring, j0, m);
        out += j0;
    }
    if (active && !active[s]) return;
    const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < m; j += gridDim.x * wpb) {
        int K = -1;
        for (int sl = slice0[s] + lane; sl < slice0[s + 1]; sl += 32)
            K = max(K, (int)out1[((uint64_t)sl * m + j) * 5 + 4]);
        K = __reduce_max_sync(0xffffffffu, K);
        __int128 ar = 0, ai = 0;
        for (int sl = slice0[s] + lane; sl < slice0[s + 1]; sl += 32) {
            const long long *q = out1 + ((uint64_t)sl * m + j) * 5;
            const int d = K - (int)q[4];
            const __int128 vr = (__int128)(((unsigned __int128)(unsigned long long)q[1] << 64) |
                                           (unsigned long long)q[0]);
            const __int128 vi = (__int128)(((unsigned __int128)(unsigned long long)q[3] << 64) |
                                           (unsigned long long)q[2]);
            ar += align_round(vr, d);
            ai += align_round(vi, d);
        }
        ar = warp_sum_i128(ar);
        if (cx) ai = warp_sum_i128(ai);
        if (lane == 0)
            out[(uint64_t)s * ldo + j] = make_double2(i128_ldexp(ar, K - 2098), cx ? i128_ldexp(ai, K - 2098) : 0.0);
    }
}

// both levels: the per-sector dot products of the last k_dotx launch
// (nslices == S with one slice per sector, as reduce_slices reports: the
// first level writes them)
static int reducex_launch(const long long *part, long long *out1, int m, int mgrid, const int *chunk0,
                          const int *slice0, int nslices, int S, const int *active, double2 *out, int ldo,
                          cudaStream_t st, const int *dx = nullptr, int ring = 0, int cx = 1, bool one = false) {
    if (one && nslices == S && S > 0) {
        k_reducex1<<<dim3(nslices, (mgrid + 7) / 8), NTHREADS, 0, st>>>(part, m, chunk0, slice0, S, active, out1,
                                                                         dx, ring, out, ldo, cx);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    if (nslices > 0) {
        k_reducex1<<<dim3(nslices, (mgrid + 7) / 8), NTHREADS, 0, st>>>(part, m, chunk0, slice0, S, active, out1,
                                                                         dx, ring);
        QS3_LAUNCHED();
    }
    k_reducex2<<<dim3((mgrid + 7) / 8, S), NTHREADS, 0, st>>>(out1, m, slice0, active, out, ldo, dx, ring, cx);
    QS3_LAUNCHED();
    return QS3_OK;
}

// the wait-timeout injection (qs3_inject_wait_timeout): 1 while launches to
// starve remain, counting them down
int take_wait_injection();

// k_dotb's ring: one resident block per SM and six stages of complex rows
// (197 KB of shared memory), twelve of real rows (half the bytes each)
template <typename VT> constexpr int dotb_ns() { return IsC<VT>::v ? 6 : 12; }
// the shared-memory size of k_dotb (once per process, before any launch or
// capture)
template <typename VT> static int dotb_prepare() {
    static const cudaError_t e = cudaFuncSetAttribute(k_dotb<VT, dotb_ns<VT>()>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)dotb_smem<VT, dotb_ns<VT>()>());
    QS3_CUDA(e);
    return QS3_OK;
}

// The dot pass: nv = 1, 2 or 4 stored vectors per pass of k_dotx (register
// staging), or nv = 8 the copy-engine ring of k_dotb (dg must then have 16
// readable bytes past its last slot, err a device int; dotb_prepare done).
// Passes over at most two vectors (the three-term part) run k_dotx.
template <typename VT>
static int dotx_launch(int nv, const typename DigT<VT>::T *dg, const int *ge, int nchunks, uint64_t D, int j0, int m,
                       const VT *w, const SecView *secs, const int *c0, int S, const int *act, long long *pp,
                       cudaStream_t st, const int *dx = nullptr, int ring = 0, int *err = nullptr) {
    const bool small = ring || (!dx && m <= 2);
    if (nv >= 8 && !small && err) {
        k_dotb<VT, dotb_ns<VT>()><<<std::max(nchunks, 1), XT + 32, dotb_smem<VT, dotb_ns<VT>()>(), st>>>(
            dg, ge, nchunks, D, j0, m, w, secs, c0, S, act, pp, err, take_wait_injection(), dx, ring);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    // complex rows stage at most 2 vectors (4 would spill registers); a
    // one-vector pass (alpha_x's dot) stages one
    if (nv >= 8 || small || IsC<VT>::v) nv = std::min(nv, 2);
    if (ring == 2 || (!dx && m == 1)) nv = 1;
    const int g = std::max(nchunks, 1);
    if (nv == 1) {
        k_dotx<VT, 1><<<g, XT, 0, st>>>(dg, ge, nchunks, D, j0, m, w, secs, c0, S, act, pp, dx, ring);
    } else if (nv == 2) {
        k_dotx<VT, 2><<<g, XT, 0, st>>>(dg, ge, nchunks, D, j0, m, w, secs, c0, S, act, pp, dx, ring);
    } else {
        if constexpr (!IsC<VT>::v)
            k_dotx<VT, 4><<<g, XT, 0, st>>>(dg, ge, nchunks, D, j0, m, w, secs, c0, S, act, pp, dx, ring);
    }
    QS3_LAUNCHED();
    return QS3_OK;
}

// out[s * ldo + j] = sum over the chunks of sector s of part[c * m + j], one
// warp per coefficient (graph mode: the range of graph_range, written from
// out + j0)
__global__ void k_reduce64(const double2 *__restrict__ part, int m, const int *__restrict__ chunk0,
                           const int *__restrict__ active, double2 *__restrict__ out, int ldo,
                           const int *__restrict__ dx = nullptr, int ring = 0) {
    const int s = blockIdx.y;
    if (dx) {
        int j0 = 0;
        graph_range(dx, ring, j0, m);
        out += j0;
    }
    if (active && !active[s]) return;
    const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < m; j += gridDim.x * wpb) {
        double2 acc = make_double2(0.0, 0.0);
        for (int c = chunk0[s] + lane; c < chunk0[s + 1]; c += 32) {
            const double2 v = part[(uint64_t)c * m + j];
            acc.x += v.x;
            acc.y += v.y;
        }
        acc = warp_sum2(acc);
        if (lane == 0) out[(uint64_t)s * ldo + j] = acc;
    }
}

// w -= sum_j V_{j0+j} coef[s][j] (binary64 FMAs from w), and part[c] = |w|^2
// over chunk c.  With wn2 (|w|^2 before the update) and strict == 0, a sector
// whose coefficients satisfy (sum_j |re c_j| + |im c_j|)^2 <= 2^-80 |w|^2
// (times (256 / m)^2 for m > 256)
// forms the correction in fp32 from the top digits of the digit store
// instead (see the file head for the bound).  One block of XT threads per
// chunk; the fp32 pass reads UV vectors' top digits per stage, two stages in
// flight.  Graph mode (dx): the range of graph_range, and for the three-term
// pass (ring) the coefficients from coef + j0.
constexpr int UV = 4;
template <typename VT>
__global__ void __launch_bounds__(XT)
    k_upd64(VT *__restrict__ w, const typename PlS<VT>::T *__restrict__ V, const typename DigT<VT>::T *__restrict__ dg,
            const int *__restrict__ ge, int nchunks, uint64_t D, int j0, int m,
            const double2 *__restrict__ coef, int ldc, const SecView *__restrict__ secs,
            const int *__restrict__ chunk0, int S, const int *__restrict__ active, const double2 *__restrict__ wn2,
            int strict, double2 *__restrict__ part, const int *__restrict__ dx = nullptr, int ring = 0) {
    using T = typename PlS<VT>::T;
    constexpr bool CX = IsC<VT>::v;
    if (dx) {
        graph_range(dx, ring, j0, m);
        if (ring) coef += j0;
    }
    extern __shared__ double2 scd[];              // m coefficients, then m fp32 copies
    float2 *scf = (float2 *)(scd + m);
    __shared__ double red[XW];
    __shared__ int lite_s;
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double cs = 0.0;
    for (int j = threadIdx.x; j < m; j += XT) {
        const double2 c = coef[(uint64_t)ci.s * ldc + j];
        scd[j] = c;
        scf[j] = make_float2((float)c.x, (float)c.y);
        cs += fabs(c.x) + fabs(c.y);
    }
    if (m > 32) {
#pragma unroll
        for (int o = 16; o; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        if (lane == 0) red[warp] = cs;
    } else if (warp == 0) {
#pragma unroll
        for (int o = 16; o; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        if (lane == 0) red[0] = cs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        const int nw = m > 32 ? XW : 1;
        for (int q = 0; q < nw; ++q) t += red[q];
        const double lim = m > 256 ? 0x1p-80 * (256.0 / m) * (256.0 / m) : 0x1p-80;
        lite_s = (!strict && wn2 && t * t <= lim * wn2[ci.s].x) ? 1 : 0;
    }
    __syncthreads();
    const bool lite = lite_s != 0;
    const int nk = (ci.n - (int)threadIdx.x + XT - 1) / XT;
    const uint64_t r0 = ci.base + threadIdx.x;
    double nrm = 0.0;
    if (lite) {
        // stored vector j, row: psi ~ (P1 / 32) 2^(em - 1044) (floor of P1 / 32,
        // an error below 2^-21 of the warp group's largest magnitude)
        using G = typename DigT<VT>::T;
        struct Stage {
            G h[UV][XR];
            int em[UV];
        };
        float2 u[XR];
#pragma unroll
        for (int k = 0; k < XR; ++k) u[k] = make_float2(0.f, 0.f);
        auto load = [&](Stage &b, int jb) {
#pragma unroll
            for (int v = 0; v < UV; ++v) {
                const int j = j0 + min(jb + v, m - 1);
                const G *slot = dg + (uint64_t)j * 2 * D;
                b.em[v] = ge[((uint64_t)j * nchunks + blockIdx.x) * XW + warp];
#pragma unroll
                for (int k = 0; k < XR; ++k) b.h[v][k] = k < nk ? slot[r0 + (uint64_t)k * XT] : G{};
            }
        };
        auto consume = [&](const Stage &b, int jb) {
#pragma unroll
            for (int v = 0; v < UV; ++v) {
                if (jb + v < m) {
                    // the coefficient times the group's scale 2^(em - 1044) (0 below
                    // the fp32 range: those values are under 2^-104)
                    const int ex = b.em[v] - 1044 + 127;
                    const float sc = (ex >= 1 && ex <= 254) ? __int_as_float(ex << 23) : 0.f;
                    const float2 c0 = scf[jb + v];
                    const float2 c = make_float2(c0.x * sc, c0.y * sc);
#pragma unroll
                    for (int k = 0; k < XR; ++k) {
                        // u += a c: re += a.r c.r - a.i c.i ; im += a.r c.i + a.i c.r
                        const float2 a = p1_f2(b.h[v][k]);
                        u[k].x = fmaf(a.x, c.x, u[k].x);
                        if (CX) {
                            u[k].x = fmaf(-a.y, c.y, u[k].x);
                            u[k].y = fmaf(a.x, c.y, u[k].y);
                            u[k].y = fmaf(a.y, c.x, u[k].y);
                        }
                    }
                }
            }
        };
        Stage s0, s1;
        if (m > 0) load(s0, 0);
#pragma unroll 1
        for (int jb = 0; jb < m; jb += 2 * UV) {
            if (jb + UV < m) load(s1, jb + UV);
            consume(s0, jb);
            if (jb + UV >= m) break;
            if (jb + 2 * UV < m) load(s0, jb + 2 * UV);
            consume(s1, jb + UV);
        }
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            if (k < nk) {
                const uint64_t r = r0 + (uint64_t)k * XT;
                double2 v = ld2(w + r);
                v.x -= (double)u[k].x;
                if (CX) v.y -= (double)u[k].y;
                st2(w + r, v);
                nrm = fma(v.x, v.x, nrm);
                if (CX) nrm = fma(v.y, v.y, nrm);
            }
        }
    } else {
        double2 acc[XR];
#pragma unroll
        for (int k = 0; k < XR; ++k) acc[k] = k < nk ? ld2(w + r0 + (uint64_t)k * XT) : make_double2(0.0, 0.0);
#pragma unroll 2
        for (int j = 0; j < m; ++j) {
            const double2 c = scd[j];
            const T *slot = V + (uint64_t)(j0 + j) * 2 * D;
#pragma unroll
            for (int k = 0; k < XR; ++k) {
                if (k < nk) {
                    const double2 a = pl_ld(slot, D, r0 + (uint64_t)k * XT);
                    // w -= a c: re -= a.r c.r - a.i c.i ; im -= a.r c.i + a.i c.r
                    acc[k].x = fma(-a.x, c.x, acc[k].x);
                    if (CX) {
                        acc[k].x = fma(a.y, c.y, acc[k].x);
                        acc[k].y = fma(-a.x, c.y, acc[k].y);
                        acc[k].y = fma(-a.y, c.x, acc[k].y);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            if (k < nk) {
                st2(w + r0 + (uint64_t)k * XT, acc[k]);
                nrm = fma(acc[k].x, acc[k].x, nrm);
                if (CX) nrm = fma(acc[k].y, acc[k].y, nrm);
            }
        }
    }
    if (part) {
#pragma unroll
        for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        __syncthreads();                          // red is reused
        if (lane == 0) red[warp] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < XW; ++q) t += red[q];
            part[blockIdx.x] = make_double2(t, 0.0);
        }
    }
}

// a float as a double, exactly, in integer instructions (the conversion
// instruction runs on the fp64 pipe): a normal float moves its exponent and
// significand into place; zero, subnormals, inf and NaN take the conversion
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// |x| with its significand truncated to 24 bits, as a float (0 below the
// normal fp32 range and above 2^54, where the square would leave the fp32
// range): never above |x|
__device__ __forceinline__ float f_trunc_abs(double x) {
    const int hi = __double2hiint(x);
    const int e = ((hi >> 20) & 0x7ff) - 896;               // the float's biased exponent
    if (e <= 0 || e > 181) return 0.f;
    return __int_as_float((e << 23) | ((hi & 0xfffff) << 3) | ((unsigned)__double2loint(x) >> 29));
}

// The three-term part of step x (Alg. 10): w -= beta_{x-1} psi_{x-1} +
// alpha_x psi_x with the recurrence's real scalars -- alpha_x the real part
// of the dot psi_x^H w in h[s][x], beta_{x-1} from the previous step (none
// for x = 0); what remains of w along psi_x and psi_{x-1} (the imaginary
// part of the dot, rounding) goes to the Gram-Schmidt pass -- in binary64
// FMAs (psi_{x-1} first), and part[c] = a lower estimate of |w|^2 over chunk
// c (values truncated to 24 bits, squared and summed in fp32, the sum lowered
// by 2^-18 of itself): it only feeds the test of the fp32 Gram-Schmidt
// correction, which a low |w| makes stricter.  Two blocks per SM, so that one
// block's FMAs (the fp64 pipe is the bound) overlap another's loads.  Graph
// mode (dx): x = *dx.
template <typename VT>
__global__ void __launch_bounds__(XT, 2)
    k_upd3(VT *__restrict__ w, const typename PlS<VT>::T *__restrict__ V, uint64_t D, int x,
           const double2 *__restrict__ h, const double *__restrict__ beta, int cap, const SecView *__restrict__ secs,
           const int *__restrict__ chunk0, int S, const int *__restrict__ active, double2 *__restrict__ part,
           const int *__restrict__ dx = nullptr) {
    using T = typename PlS<VT>::T;
    constexpr bool CX = IsC<VT>::v;
    if (dx) x = *dx;
    __shared__ float red[XW];
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (ci.n - (int)threadIdx.x + XT - 1) / XT;
    const uint64_t r0 = ci.base + threadIdx.x;
    double2 acc[XR], p[XR], q[XR];
    const T *sp = V + (uint64_t)(x > 0 ? x - 1 : 0) * 2 * D, *sq = V + (uint64_t)x * 2 * D;
#pragma unroll
    for (int k = 0; k < XR; ++k) {
        const bool in = k < nk;
        const uint64_t r = r0 + (uint64_t)k * XT;
        acc[k] = in ? ld2(w + r) : make_double2(0.0, 0.0);
        p[k] = (in && x > 0) ? pl_ld(sp, D, r) : make_double2(0.0, 0.0);
        q[k] = in ? pl_ld(sq, D, r) : make_double2(0.0, 0.0);
    }
    const double a = h[(uint64_t)ci.s * cap + x].x;
    const double b = x > 0 ? beta[(uint64_t)ci.s * cap + x - 1] : 0.0;
    float nf = 0.f;
#pragma unroll
    for (int k = 0; k < XR; ++k) {
        if (k < nk) {
            if (x > 0) {
                acc[k].x = fma(-p[k].x, b, acc[k].x);
                if (CX) acc[k].y = fma(-p[k].y, b, acc[k].y);
            }
            acc[k].x = fma(-q[k].x, a, acc[k].x);
            if (CX) acc[k].y = fma(-q[k].y, a, acc[k].y);
            st2(w + r0 + (uint64_t)k * XT, acc[k]);
            const float fx = f_trunc_abs(acc[k].x);
            nf = fmaf(fx, fx, nf);
            if (CX) {
                const float fy = f_trunc_abs(acc[k].y);
                nf = fmaf(fy, fy, nf);
            }
        }
    }
    if (part) {
#pragma unroll
        for (int o = 16; o; o >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, o);
        if (lane == 0) red[warp] = nf;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int qq = 0; qq < XW; ++qq) t += (double)red[qq];
            part[blockIdx.x] = make_double2(t * (1.0 - 0x1p-18), 0.0);
        }
    }
}

// The Gram-Schmidt update with the stored vectors' top digits brought in by
// TMA bulk copies (k_updb): the arithmetic of k_upd64 (the same lite test,
// the fp32 correction from the P1 digits summed in the same order, w - u in
// binary64; the binary64 FMA path when the test fails), with a copy warp
// (warp XW) filling a ring of ns stages, each the chunk's slice of the P1
// plane of one stored vector (from the 16-byte boundary at or below the
// chunk, rounded up to 16 bytes) and its XW group exponents.  Dynamic shared
// memory: the ring, then the m coefficients and their fp32 copies.  Waits
// are bounded as in k_dotb (a wait that runs out sets *err; the block still
// writes w and its norm, both finite).  starve != 0: the copy warp issues
// nothing (the test injection).  Graph mode (dx): the range of graph_range.
constexpr int UB_NSMAX = 24;
constexpr int UPDB_SMEM = 110 * 1024;          // dynamic shared memory per block (two blocks per SM)
template <typename VT> constexpr unsigned updb_stage() { return dotb_slice<VT>() + XW * 4; }

__device__ __forceinline__ void bar_consumers() { asm volatile("bar.sync 1, %0;" ::"r"(XT) : "memory"); }

template <typename VT>
__global__ void __launch_bounds__(XT + 32, 2)
    k_updb(VT *__restrict__ w, const typename PlS<VT>::T *__restrict__ V, const typename DigT<VT>::T *__restrict__ dg,
           const int *__restrict__ ge, int nchunks, uint64_t D, int j0, int m, int ns,
           const double2 *__restrict__ coef, int ldc, const SecView *__restrict__ secs,
           const int *__restrict__ chunk0, int S, const int *__restrict__ active, const double2 *__restrict__ wn2,
           double2 *__restrict__ part, int *__restrict__ err, int starve, const int *__restrict__ dx = nullptr) {
    using G = typename DigT<VT>::T;
    using T = typename PlS<VT>::T;
    constexpr bool CX = IsC<VT>::v;
    constexpr unsigned SL = dotb_slice<VT>(), SB = updb_stage<VT>();
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[UB_NSMAX], empty[UB_NSMAX];
    __shared__ double red[XW];
    __shared__ int lite_s;
    graph_range(dx, 0, j0, m);
    double2 *scd = (double2 *)(dsm + (size_t)ns * SB);
    float2 *scf = (float2 *)(scd + m);
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int t = 0; t < ns; ++t) {
            mbar_init(&full[t], 1);
            mbar_init(&empty[t], XW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the copy warp fills the first stages at once (most passes take the fp32
    // correction) and the consumers fetch their rows of w, both while the
    // coefficients are read and the test below is taken
    auto plane1 = [&](int jj) { return dg + (uint64_t)(j0 + jj) * 2 * D + ci.base; };
    const unsigned nb = (unsigned)ci.n * (unsigned)sizeof(G);
    int issued = 0;
    auto issue = [&](int t) {
        unsigned char *sp = dsm + (size_t)t * SB;
        const G *p1 = plane1(issued);
        const unsigned o1 = (unsigned)((uintptr_t)p1 & 15u);
        const unsigned b1 = (o1 + nb + 15u) & ~15u;
        mbar_expect_tx(&full[t], b1 + XW * 4);
        bulk_g2s(sp, (const unsigned char *)p1 - o1, b1, &full[t]);
        bulk_g2s(sp + SL, ge + ((uint64_t)(j0 + issued) * nchunks + blockIdx.x) * XW, XW * 4, &full[t]);
        ++issued;
    };
    if (warp == XW && lane == 0 && wn2 && !starve)
        while (issued < m && issued < ns) issue(issued);
    const int nk = (ci.n - (int)threadIdx.x + XT - 1) / XT;
    const uint64_t r0 = ci.base + threadIdx.x;
    double2 wr[XR];
    // the coefficients, their fp32 copies and the lite test (as k_upd64)
    if (warp < XW) {
#pragma unroll
        for (int k = 0; k < XR; ++k) wr[k] = k < nk ? ld2(w + r0 + (uint64_t)k * XT) : make_double2(0.0, 0.0);
        double cs = 0.0;
        for (int j = threadIdx.x; j < m; j += XT) {
            const double2 c = coef[(uint64_t)ci.s * ldc + j];
            scd[j] = c;
            scf[j] = make_float2((float)c.x, (float)c.y);
            cs += fabs(c.x) + fabs(c.y);
        }
        if (m > 32) {
#pragma unroll
            for (int o = 16; o; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
            if (lane == 0) red[warp] = cs;
        } else if (warp == 0) {
#pragma unroll
            for (int o = 16; o; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
            if (lane == 0) red[0] = cs;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        const int nw = m > 32 ? XW : 1;
        for (int q = 0; q < nw; ++q) t += red[q];
        const double lim = m > 256 ? 0x1p-80 * (256.0 / m) * (256.0 / m) : 0x1p-80;
        lite_s = (wn2 && t * t <= lim * wn2[ci.s].x) ? 1 : 0;
    }
    __syncthreads();
    const bool lite = lite_s != 0;
    if (warp == XW) {
        // the copy warp: the rest of the ring for the fp32 correction; the
        // binary64 path reads no digits (the stages in flight land first)
        if (lane == 0) {
            bool ok = true;
            int t = issued % ns;
            unsigned q = (unsigned)(issued / ns - 1) & 1u;     // parity of the empty phase to wait for
            for (; lite && issued < m && !starve;) {
                if (!mbar_wait(&empty[t], q)) {
                    ok = false;
                    break;
                }
                fence_proxy_async();
                issue(t);
                if (++t == ns) {
                    t = 0;
                    q ^= 1u;
                }
            }
            if (!ok) atomicExch(err, 1);
            for (int jj = issued - ns > 0 ? issued - ns : 0; jj < issued; ++jj)
                mbar_wait(&full[jj % ns], (unsigned)(jj / ns) & 1u);
        }
        return;
    }
    double nrm = 0.0;
    if (lite) {
        // stored vector j, row: psi ~ (P1 / 32) 2^(em - 1044), as in k_upd64
        const unsigned ob1 = (unsigned)((uintptr_t)plane1(0) & 15u);
        const unsigned osl = (unsigned)(2 * D * sizeof(G)) & 15u;
        float2 u[XR];
#pragma unroll
        for (int k = 0; k < XR; ++k) u[k] = make_float2(0.f, 0.f);
        // two stored vectors per pass; the stage index t and the phase parity
        // q advance with the pass (no division by the runtime ring depth)
        auto corr = [&](const G (&h)[XR], int em, int jj) {
            const int ex = em - 1044 + 127;
            const float sc = (ex >= 1 && ex <= 254) ? __int_as_float(ex << 23) : 0.f;
            const float2 c0 = scf[jj];
            const float2 c = make_float2(c0.x * sc, c0.y * sc);
#pragma unroll
            for (int k = 0; k < XR; ++k) {
                const float2 a = p1_f2(h[k]);
                u[k].x = fmaf(a.x, c.x, u[k].x);
                if (CX) {
                    u[k].x = fmaf(-a.y, c.y, u[k].x);
                    u[k].y = fmaf(a.x, c.y, u[k].y);
                    u[k].y = fmaf(a.y, c.x, u[k].y);
                }
            }
        };
        int t = 0;
        unsigned q = 0;
#pragma unroll 1
        for (int jj = 0; jj < m; jj += 2) {
            const bool two = jj + 1 < m;
            const int t1 = t + 1 == ns ? 0 : t + 1;
            const unsigned q1 = t + 1 == ns ? q ^ 1u : q;
            bool ok = true;
            if (lane == 0) {
                ok = mbar_wait(&full[t], q);
                if (ok && two) ok = mbar_wait(&full[t1], q1);
            }
            if (!__shfl_sync(0xffffffffu, (int)ok, 0)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            mbar_try(&full[t], q);
            if (two) mbar_try(&full[t1], q1);
            const unsigned char *s0 = dsm + (size_t)t * SB, *s1 = dsm + (size_t)t1 * SB;
            const G *pa = (const G *)(s0 + ((ob1 + (unsigned)jj * osl) & 15u));
            const G *pb = (const G *)(s1 + ((ob1 + (unsigned)(jj + 1) * osl) & 15u));
            G h0[XR], h1[XR];
#pragma unroll
            for (int k = 0; k < XR; ++k) {
                h0[k] = k < nk ? pa[threadIdx.x + k * XT] : G{};
                h1[k] = (two && k < nk) ? pb[threadIdx.x + k * XT] : G{};
            }
            const int em0 = ((const int *)(s0 + SL))[warp];
            const int em1 = two ? ((const int *)(s1 + SL))[warp] : 0;
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[t]);
                if (two) mbar_arrive(&empty[t1]);
            }
            corr(h0, em0, jj);
            if (two) corr(h1, em1, jj + 1);
            t = t1 + 1 == ns ? 0 : t1 + 1;
            q = t1 + 1 == ns ? q1 ^ 1u : q1;
        }
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            if (k < nk) {
                const uint64_t r = r0 + (uint64_t)k * XT;
                double2 v = wr[k];
                v.x -= f2d_exact(u[k].x);
                if (CX) v.y -= f2d_exact(u[k].y);
                st2(w + r, v);
                nrm = fma(v.x, v.x, nrm);
                if (CX) nrm = fma(v.y, v.y, nrm);
            }
        }
    } else {
        double2 acc[XR];
#pragma unroll
        for (int k = 0; k < XR; ++k) acc[k] = wr[k];
#pragma unroll 2
        for (int j = 0; j < m; ++j) {
            const double2 c = scd[j];
            const T *slot = V + (uint64_t)(j0 + j) * 2 * D;
#pragma unroll
            for (int k = 0; k < XR; ++k) {
                if (k < nk) {
                    const double2 a = pl_ld(slot, D, r0 + (uint64_t)k * XT);
                    acc[k].x = fma(-a.x, c.x, acc[k].x);
                    if (CX) {
                        acc[k].x = fma(a.y, c.y, acc[k].x);
                        acc[k].y = fma(-a.x, c.y, acc[k].y);
                        acc[k].y = fma(-a.y, c.x, acc[k].y);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < XR; ++k) {
            if (k < nk) {
                st2(w + r0 + (uint64_t)k * XT, acc[k]);
                nrm = fma(acc[k].x, acc[k].x, nrm);
                if (CX) nrm = fma(acc[k].y, acc[k].y, nrm);
            }
        }
    }
    if (part) {
#pragma unroll
        for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        bar_consumers();                          // red is reused
        if (lane == 0) red[warp] = nrm;
        bar_consumers();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < XW; ++q) t += red[q];
            part[blockIdx.x] = make_double2(t, 0.0);
        }
    }
}

// the ring depth of k_updb for up to mmax coefficients (0: k_upd64 instead)
template <typename VT> static int updb_ns(int mmax) {
    const long long ns = ((long long)UPDB_SMEM - (long long)mmax * 24) / (long long)updb_stage<VT>();
    return ns >= 2 ? (int)std::min<long long>(ns, UB_NSMAX) : 0;
}
template <typename VT> static int updb_prepare() {
    static const cudaError_t e =
        cudaFuncSetAttribute(k_updb<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, UPDB_SMEM);
    QS3_CUDA(e);
    return QS3_OK;
}

// psi_{x+1} = w * inv[s]: into the store's slot (graph mode: slot *dx + 1 of
// the store at out), its digit-store image (dg, ge) and hin, the interleaved
// input of the next H Phi.  w may alias hin (the start vector is normalised
// in place).  One block of XT threads per chunk.
template <typename VT>
__global__ void __launch_bounds__(XT)
    k_scale64(const VT *w, typename PlS<VT>::T *__restrict__ out, typename DigT<VT>::T *__restrict__ dg,
              int *__restrict__ ge, int nchunks, VT *hin, const double *__restrict__ inv,
              const SecView *__restrict__ secs, const int *__restrict__ chunk0, int S, const int *__restrict__ active,
              const int *__restrict__ dx, uint64_t D) {
    constexpr int NC = IsC<VT>::v ? 2 : 1;
    if (dx) {
        out += (uint64_t)(*dx + 1) * 2 * D;
        dg += (uint64_t)(*dx + 1) * 2 * D;
        ge += (uint64_t)(*dx + 1) * nchunks * XW;
    }
    const ChunkInfo ci = chunk_info(secs, chunk0, S, blockIdx.x);
    if (active && !active[ci.s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double f = inv[ci.s];
    uint32_t hw[XR][2], lw[XR][2];
#pragma unroll
    for (int k = 0; k < XR; ++k) {
        const int r = threadIdx.x + k * XT;
        double2 v = make_double2(0.0, 0.0);
        if (r < ci.n) {
            v = ld2(w + ci.base + r);
            v.x *= f;
            v.y *= f;
            pl_st(out, D, ci.base + r, v);
            st2(hin + ci.base + r, v);
        }
        hw[k][0] = (uint32_t)__double2hiint(v.x);
        lw[k][0] = (uint32_t)__double2loint(v.x);
        hw[k][1] = (uint32_t)__double2hiint(v.y);
        lw[k][1] = (uint32_t)__double2loint(v.y);
    }
    int d1[XR][2], d0[XR][2];
    const int em = fx_group<NC>(hw, lw, d1, d0);
#pragma unroll
    for (int k = 0; k < XR; ++k) {
        const int r = threadIdx.x + k * XT;
        if (r < ci.n) dig_st(dg, D, ci.base + r, d1[k], d0[k]);
    }
    if (lane == 0) ge[(uint64_t)blockIdx.x * XW + warp] = em;
}

// out_y[r] = sum_x V_x[r] C[s][x][y] (binary64 FMAs), y < nout <= MAXOUT, for
// the rows of sectors with mask[s] != 0.  PLO: out is the store (output y in
// slot y of out); else out holds interleaved fp64 vectors ldo apart.
template <typename VT, bool PLO>
__global__ void __launch_bounds__(NTHREADS)
    k_comb64(void *__restrict__ outp, uint64_t ldo, const typename PlS<VT>::T *__restrict__ V, uint64_t D, int nin,
             int nout, const double *__restrict__ C, int ldc, const SecView *__restrict__ secs,
             const int *__restrict__ chunk0, int S, const int *__restrict__ mask) {
    using T = typename PlS<VT>::T;
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
    if (nout == 1) {
        // one output: each thread's rows in registers, all their loads of a
        // stored vector in flight together
        const int nk = (ci.n - (int)threadIdx.x + NTHREADS - 1) / NTHREADS;
        const uint64_t r0 = ci.base + threadIdx.x;
        double2 acc[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[k] = make_double2(0.0, 0.0);
        for (int x = 0; x < nin; ++x) {
            const double c = sc[x];
            const T *slot = V + (uint64_t)x * 2 * D;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (k < nk) {
                    const double2 a = pl_ld(slot, D, r0 + (uint64_t)k * NTHREADS);
                    acc[k].x = fma(a.x, c, acc[k].x);
                    acc[k].y = fma(a.y, c, acc[k].y);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (k < nk) {
                const uint64_t r = r0 + (uint64_t)k * NTHREADS;
                if constexpr (PLO) pl_st((T *)outp, D, r, acc[k]);
                else st2((VT *)outp + r, acc[k]);
            }
        }
        return;
    }
#pragma unroll 1
    for (int k = 0; k < RPT; ++k) {
        const int r = threadIdx.x + k * NTHREADS;
        if (r >= ci.n) continue;
        double2 acc[MAXOUT];
#pragma unroll
        for (int y = 0; y < MAXOUT; ++y) acc[y] = make_double2(0.0, 0.0);
        for (int x = 0; x < nin; ++x) {
            const double2 a = pl_ld(V + (uint64_t)x * 2 * D, D, ci.base + r);
#pragma unroll
            for (int y = 0; y < MAXOUT; ++y)
                if (y < nout) {
                    const double c = sc[x * nout + y];
                    acc[y].x = fma(a.x, c, acc[y].x);
                    acc[y].y = fma(a.y, c, acc[y].y);
                }
        }
#pragma unroll
        for (int y = 0; y < MAXOUT; ++y)
            if (y < nout) {
                if constexpr (PLO) pl_st((T *)outp + (uint64_t)y * 2 * D, D, ci.base + r, acc[y]);
                else st2((VT *)outp + (uint64_t)y * ldo + ci.base + r, acc[y]);
            }
    }
}

// ------------------------------------------------------------------ engine
template <typename VT>
struct Engine64 {
    using WT = VT;                         // result vectors are binary64 as well
    using ST = typename PlS<VT>::T;        // word of the planar store
    Basis &B;
    cudaStream_t st;
    HphiStats *stats;
    int cap = 0, nscr = 0;
    uint64_t D = 0;
    DevBuf V, DG, GE, wbuf, hinb, part, partx, partr, slices, h1, h2, alpha, beta, nrm, nrm1, inv, active, derr;
    int nslices = 0;
    bool slice1 = false;                   // one reduction slice per sector
    std::vector<int> h_active;
    double brk = 1e-12;
    int strict = 0;                        // 1: every update on binary64 FMAs
    bool graphs = false;
    DevBuf xdev;
    int xdev_val = -1;
    cudaStream_t cs = nullptr;
    cudaGraphExec_t gx = nullptr;
    long long gnodes = 0;

    Engine64(Basis &b, cudaStream_t s, HphiStats *hs) : B(b), st(s), stats(hs) {}
    ~Engine64() {
        if (gx) cudaGraphExecDestroy(gx);
        if (cs) cudaStreamDestroy(cs);
    }
    Engine64(const Engine64 &) = delete;
    Engine64 &operator=(const Engine64 &) = delete;
    void use_df_hphi(bool) {}
    void set_strict(bool on) { strict = on ? 1 : 0; }
    bool loop_graph_ok() const { return graphs; }
    int enable_graphs(bool on) {
        graphs = on && B.nchunks > 0;
        if (graphs && !xdev.p) QS3_TRY(xdev.alloc(sizeof(int)));
        return QS3_OK;
    }
    qs3_dtype dtype() const { return IsC<VT>::v ? QS3_C128 : QS3_F64; }
    // slot j of the store (2 D words-per-element units)
    ST *svec(int j) { return V.as<ST>() + (uint64_t)j * 2 * D; }
    // the digit store: slot j's digits and its grid exponents
    typename DigT<VT>::T *dg(int j = 0) { return DG.as<typename DigT<VT>::T>() + (uint64_t)j * 2 * D; }
    int *ge(int j = 0) { return GE.as<int>() + (uint64_t)j * std::max(B.nchunks, 1) * XW; }
    size_t slot_bytes() const { return (size_t)D * sizeof(VT); }
    VT *hin(int) { return hinb.as<VT>(); }
    VT *wv() { return wbuf.as<VT>(); }
    const SecView *secs() { return B.d_secs.as<SecView>(); }
    const int *c0() { return B.d_chunk0.as<int>(); }
    int *act() { return active.as<int>(); }
    int grid() const { return std::max(B.nchunks, 1); }

    int init(int cap_, int nscratch) {
        cap = cap_;
        nscr = nscratch;
        D = B.total;
        QS3_TRY(V.alloc((uint64_t)(cap + nscr) * D * sizeof(VT)));
        QS3_TRY(DG.alloc((uint64_t)(cap + nscr) * D * sizeof(VT) + 16));     // k_dotb reads up to 16 bytes past
        QS3_TRY(GE.alloc((uint64_t)(cap + nscr) * std::max(B.nchunks, 1) * XW * sizeof(int)));
        QS3_TRY(wbuf.alloc(std::max<uint64_t>(D, 1) * sizeof(VT)));
        QS3_TRY(hinb.alloc(std::max<uint64_t>(D, 1) * sizeof(VT)));
        QS3_TRY(part.alloc((uint64_t)std::max(B.nchunks, 1) * cap * sizeof(double2)));
        QS3_TRY(partx.alloc((uint64_t)std::max(B.nchunks, 1) * cap * XW * 3 * sizeof(long long)));
        {
            const std::vector<int> s0 = reduce_slices(B);
            nslices = s0[B.S];
            slice1 = one_slice(s0);
            QS3_TRY(slices.upload(s0.data(), s0.size() * sizeof(int)));
            QS3_TRY(partr.alloc((uint64_t)std::max(nslices, 1) * cap * 5 * sizeof(long long)));
        }
        QS3_TRY(h1.alloc((uint64_t)B.S * cap * sizeof(double2)));
        QS3_TRY(h2.alloc((uint64_t)B.S * cap * sizeof(double2)));
        QS3_TRY(alpha.alloc((uint64_t)B.S * cap * sizeof(double)));
        QS3_TRY(beta.alloc((uint64_t)B.S * cap * sizeof(double)));
        QS3_TRY(nrm.alloc((uint64_t)B.S * sizeof(double2)));
        QS3_TRY(nrm1.alloc((uint64_t)B.S * sizeof(double2)));
        QS3_TRY(inv.alloc((uint64_t)B.S * sizeof(double)));
        QS3_TRY(active.alloc((uint64_t)B.S * sizeof(int)));
        QS3_TRY(derr.alloc(sizeof(int)));
        QS3_CUDA(cudaMemsetAsync(derr.p, 0, sizeof(int), st));
        QS3_TRY(dotb_prepare<VT>());
        QS3_TRY(updb_prepare<VT>());
        QS3_CUDA(cudaMemsetAsync(alpha.p, 0, alpha.n, st));
        QS3_CUDA(cudaMemsetAsync(beta.p, 0, beta.n, st));
        h_active.assign(B.S, 0);
        for (int s = 0; s < B.S; ++s) h_active[s] = B.dims[s] > 0;
        QS3_TRY(push_active());
        return tune_dots();
    }
    // QS3_ERR_TIMEOUT if a bounded device wait of the dot pass ran out
    // (synchronises the stream)
    int check_err() {
        int e = 0;
        QS3_CUDA(cudaMemcpyAsync(&e, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaStreamSynchronize(st));
        if (e) return set_err(QS3_ERR_TIMEOUT, "a wait of the dot pass (k_dotb) ran out");
        return QS3_OK;
    }
    int push_active() {
        QS3_CUDA(cudaMemcpyAsync(active.p, h_active.data(), B.S * sizeof(int), cudaMemcpyHostToDevice, st));
        return QS3_OK;
    }
    bool any_active() const {
        for (int a : h_active) if (a) return true;
        return false;
    }
    int reduce(int m, double2 *out, int ldo, const int *dx = nullptr, int ring = 0, int mgrid = 0) {
        const int mg = mgrid > 0 ? mgrid : m;
        k_reduce64<<<dim3((mg + 7) / 8, B.S), NTHREADS, 0, st>>>(part.as<double2>(), m, c0(), act(), out, ldo, dx,
                                                                 ring);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    // the dot products of w against stored vectors j0 .. j0 + m - 1 as chunk
    // partials: k_dotx with nv stored vectors per pass (1, 2 or 4), or under
    // strict64 k_dot64 (binary64 FMA chains); dot_reduce sums them per sector
    int dot_launch(int nv, int j0, int m, const int *dx = nullptr, int ring = 0) {
        const ST *v = V.as<ST>();
        const VT *w = wv();
        if (!strict)
            return dotx_launch<VT>(nv, dg(), ge(), B.nchunks, D, j0, m, w, secs(), c0(), B.S, act(),
                                   partx.as<long long>(), st, dx, ring, derr.as<int>());
        k_dot64<VT, 2><<<grid(), NTHREADS, 0, st>>>(v, D, j0, m, w, secs(), c0(), B.S, act(), part.as<double2>(), dx,
                                                     ring);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    int dot_reduce(int m, double2 *out, int ldo, const int *dx = nullptr, int ring = 0, int mgrid = 0) {
        if (strict) return reduce(m, out, ldo, dx, ring, mgrid);
        return reducex_launch(partx.as<long long>(), partr.as<long long>(), m, mgrid > 0 ? mgrid : m, c0(),
                              slices.as<int>(), nslices, B.S, act(), out, ldo, st, dx, ring, IsC<VT>::v ? 1 : 0,
                              slice1);
    }
    // dot products of w against stored vectors j0 .. j0 + m - 1 into out (S x ldo)
    int mdot(int j0, int m, double2 *out, int ldo) {
        if (B.nchunks == 0) return QS3_OK;
        QS3_TRY(dot_launch(B.tune_nv64 > 0 ? B.tune_nv64 : 2, j0, m));
        return dot_reduce(m, out, ldo);
    }
    // the dot pass: time k_dotx with 1, 2 and 4 vectors per pass and the
    // k_dotb ring (8) on min(cap, 48) zeroed slots and keep the fastest
    // for this basis
    int tune_dots() {
        if (B.tune_nv64 != 0 || B.nchunks == 0) return QS3_OK;
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        QS3_CUDA(cudaStreamIsCapturing(st, &cst));
        if (cst != cudaStreamCaptureStatusNone) return QS3_OK;
        const int m = std::min(cap, 48);
        QS3_CUDA(cudaMemsetAsync(V.p, 0, (size_t)m * slot_bytes(), st));
        QS3_CUDA(cudaMemsetAsync(DG.p, 0, (size_t)m * slot_bytes(), st));
        QS3_CUDA(cudaMemsetAsync(GE.p, 0, (size_t)m * B.nchunks * XW * sizeof(int), st));
        QS3_CUDA(cudaMemsetAsync(wbuf.p, 0, wbuf.n, st));
        cudaEvent_t e0, e1;
        QS3_CUDA(cudaEventCreate(&e0));
        QS3_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        int bnv = 2, rc = QS3_OK;
        for (int nv : {1, 2, 4, 8}) {
            float tmin = 1e30f;
            for (int rep = 0; rep < 4 && rc == QS3_OK; ++rep) {
                if (cudaEventRecord(e0, st) != cudaSuccess) { rc = QS3_ERR_CUDA; break; }
                rc = dot_launch(nv, 0, m);
                if (rc != QS3_OK) break;
                if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = QS3_ERR_CUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tmin = std::min(tmin, ms);
            }
            if (tmin < best) { best = tmin; bnv = nv; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != QS3_OK) return set_err(rc, "dot-product autotuning failed");
        B.tune_nv64 = bnv;
        return QS3_OK;
    }
    // the Gram-Schmidt update runs k_updb (the copy ring) with the copy-ring
    // dot pass (dot_vectors64 = 8), when the fp32 correction is possible
    // (wn2 given, strict64 off), the pass is longer than the three-term one
    // and the ring fits beside mmax coefficients
    bool updb_ok(const double2 *wn2, int m, int mmax) const {
        return B.tune_nv64 == 8 && !strict && wn2 && m > 2 && updb_ns<VT>(mmax) > 0;
    }
    // w -= sum_j psi_{j0+j} cf[s][j]; nrm_out: per-sector |w|^2 after it;
    // wn2: |w|^2 before it (enables the fp32 correction of tiny coefficients)
    int mupdate(int j0, int m, const double2 *cf, int ldc, double2 *nrm_out, const double2 *wn2 = nullptr) {
        if (B.nchunks == 0) return QS3_OK;
        if (updb_ok(wn2, m, m)) {
            const int ns = updb_ns<VT>(m);
            k_updb<VT><<<grid(), XT + 32, (size_t)ns * updb_stage<VT>() + (size_t)m * 24, st>>>(
                wv(), V.as<ST>(), dg(), ge(), B.nchunks, D, j0, m, ns, cf, ldc, secs(), c0(), B.S, act(), wn2,
                part.as<double2>(), derr.as<int>(), take_wait_injection());
            QS3_LAUNCHED();
            return reduce(1, nrm_out, 1);
        }
        k_upd64<VT><<<grid(), XT, (size_t)m * (sizeof(double2) + sizeof(float2)), st>>>(
            wv(), V.as<ST>(), dg(), ge(), B.nchunks, D, j0, m, cf, ldc, secs(), c0(), B.S, act(), wn2, strict,
            part.as<double2>());
        QS3_LAUNCHED();
        return reduce(1, nrm_out, 1);
    }
    // psi_j = w * inv (per sector) into slot j and hin
    int scale_store(const VT *w, int j) {
        if (B.nchunks == 0) return QS3_OK;
        k_scale64<VT><<<grid(), XT, 0, st>>>(w, svec(j), dg(j), ge(j), B.nchunks, hin(0), inv.as<double>(), secs(),
                                             c0(), B.S, act(), nullptr, D);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    // normalise the start vector in hin per sector and store it as psi_0
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
    void count_hphi() {
        stats->calls += 1;
        for (int s = 0; s < B.S; ++s)
            if (h_active[s]) stats->nnz += B.nnz_sec[s];
    }
    // w = H psi_x: on the integer units from the digit image of slot x (slot
    // *dx in graph mode) when the basis allows it and strict64 is off, else
    // the binary64 FMA kernels
    int hphi_apply(int x, const int *dx) {
        if (!strict && IsC<VT>::v && hphi_x_ok(B))
            return dx ? hphi_x_launch(B, hin(0), DG.p, GE.as<int>(), dx, wv(), st, act())
                      : hphi_x_launch(B, hin(0), dg(x), ge(x), nullptr, wv(), st, act());
        return hphi_launch(B, dtype(), hin(x), wv(), st, act());
    }
    // the Gram-Schmidt dot pass against psi_0 .. psi_x, timed with events
    int gs_dots(int x) {
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        QS3_TRY(stats->pair(ev));
        QS3_CUDA(cudaEventRecord(ev.first, st));
        QS3_TRY(mdot(0, x + 1, h2.as<double2>(), cap));
        QS3_CUDA(cudaEventRecord(ev.second, st));
        stats->pend_gs.push_back(ev);
        stats->gs_calls += 1;
        uint64_t rows = 0;
        for (int s = 0; s < B.S; ++s)
            if (h_active[s]) rows += B.dims[s];
        stats->gs_bytes += rows * ((uint64_t)(x + 2) * sizeof(VT));
        stats->gs_fma += rows * (uint64_t)(x + 1) * (IsC<VT>::v ? 4 : 1);
        return QS3_OK;
    }
    // one step with every x-dependent count and offset taken from xdev (the
    // body of the captured graph; x >= 1, one Gram-Schmidt pass)
    int step_body_dev() {
        const int *dx = xdev.as<int>();
        VT *w = wv();
        double2 *hh1 = h1.as<double2>(), *n1 = nrm1.as<double2>();
        QS3_TRY(hphi_apply(0, dx));
        QS3_TRY(dot_launch(2, 0, 1, dx, 2));
        QS3_TRY(dot_reduce(1, hh1, cap, dx, 2, 1));
        k_upd3<VT><<<grid(), XT, 0, st>>>(w, V.as<ST>(), D, 0, hh1, beta.as<double>(), cap, secs(), c0(), B.S,
                                          act(), part.as<double2>(), dx);
        QS3_LAUNCHED();
        QS3_TRY(reduce(1, n1, 1));
        QS3_TRY(dot_launch(B.tune_nv64 > 0 ? B.tune_nv64 : 2, 0, cap, dx, 0));
        QS3_TRY(dot_reduce(cap, h2.as<double2>(), cap, dx, 0, cap));
        if (updb_ok(n1, cap, cap)) {
            const int ns = updb_ns<VT>(cap);
            k_updb<VT><<<grid(), XT + 32, (size_t)ns * updb_stage<VT>() + (size_t)cap * 24, st>>>(
                w, V.as<ST>(), dg(), ge(), B.nchunks, D, 0, cap, ns, h2.as<double2>(), cap, secs(), c0(), B.S, act(),
                n1, part.as<double2>(), derr.as<int>(), take_wait_injection(), dx);
        } else {
            k_upd64<VT><<<grid(), XT, (size_t)cap * (sizeof(double2) + sizeof(float2)), st>>>(
                w, V.as<ST>(), dg(), ge(), B.nchunks, D, 0, cap, h2.as<double2>(), cap, secs(), c0(), B.S, act(), n1,
                strict, part.as<double2>(), dx, 0);
        }
        QS3_LAUNCHED();
        QS3_TRY(reduce(1, nrm.as<double2>(), 1));
        k_step_scalars<<<(B.S + 127) / 128, 128, 0, st>>>(B.S, 0, cap, hh1, nrm.as<double2>(), act(),
                                                         alpha.as<double>(), beta.as<double>(), inv.as<double>(), brk,
                                                         dx);
        QS3_LAUNCHED();
        k_scale64<VT><<<grid(), XT, 0, st>>>(w, V.as<ST>(), dg(), ge(), B.nchunks, hin(0), inv.as<double>(), secs(),
                                             c0(), B.S, act(), dx, D);
        QS3_LAUNCHED();
        k_advance<<<1, 1, 0, st>>>(xdev.as<int>());
        QS3_LAUNCHED();
        return QS3_OK;
    }
    int graph_step(int x) {
        if (!cs) QS3_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        if (!gx) {
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
            const cudaError_t ei = cudaGraphInstantiate(&gx, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                gx = nullptr;
                return set_err(QS3_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
            }
            gnodes = (long long)nn;
            count_launch(-(long long)nn);   // the capture ran nothing
        }
        if (xdev_val != x) {
            k_setx<<<1, 1, 0, st>>>(xdev.as<int>(), x);
            QS3_LAUNCHED();
        }
        QS3_CUDA(cudaGraphLaunch(gx, st));
        count_launch(gnodes);
        xdev_val = x + 1;
        return QS3_OK;
    }
    // Alg. 10 lines 5-11 for step x (full2: the first step after a thick
    // restart, whose w has the arrowhead components beta_y psi_y: the first
    // pass then runs against all of psi_0 .. psi_x)
    int step(int x, bool full2 = false) {
        if (graphs && !full2 && x >= 1) {
            stats->graph_calls += 1;
            count_hphi();
            return graph_step(x);
        }
        VT *w = wv();
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        QS3_TRY(stats->pair(ev));
        QS3_CUDA(cudaEventRecord(ev.first, st));
        QS3_TRY(hphi_apply(x, nullptr));
        QS3_CUDA(cudaEventRecord(ev.second, st));
        stats->pend.push_back(ev);
        count_hphi();
        double2 *n1 = nrm1.as<double2>();
        if (full2) {
            // after a thick restart: a full first pass with complex coefficients
            QS3_TRY(mdot(0, x + 1, h1.as<double2>(), cap));
            QS3_TRY(mupdate(0, x + 1, h1.as<double2>(), cap, n1));
        } else {
            // alpha_x = Re psi_x^H w, then w -= beta_{x-1} psi_{x-1} + alpha_x psi_x
            QS3_TRY(mdot(x, 1, h1.as<double2>() + x, cap));
            k_upd3<VT><<<grid(), XT, 0, st>>>(w, V.as<ST>(), D, x, h1.as<double2>(), beta.as<double>(), cap, secs(),
                                              c0(), B.S, act(), part.as<double2>());
            QS3_LAUNCHED();
            QS3_TRY(reduce(1, n1, 1));
        }
        QS3_TRY(gs_dots(x));
        QS3_TRY(mupdate(0, x + 1, h2.as<double2>(), cap, nrm.as<double2>(), n1));
        k_step_scalars<<<(B.S + 127) / 128, 128, 0, st>>>(B.S, x, cap, h1.as<double2>(), nrm.as<double2>(), act(),
                                                         alpha.as<double>(), beta.as<double>(), inv.as<double>(), brk);
        QS3_LAUNCHED();
        return scale_store(w, x + 1);
    }
    int fetch(std::vector<double> &a, std::vector<double> &b) {
        a.resize((size_t)B.S * cap);
        b.resize((size_t)B.S * cap);
        QS3_CUDA(cudaMemcpyAsync(a.data(), alpha.p, a.size() * 8, cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaMemcpyAsync(b.data(), beta.p, b.size() * 8, cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaStreamSynchronize(st));
        return stats->harvest();
    }
    // out_y = sum_x psi_x C[s][x][y] (x < nin, y < nout) for the sectors in
    // mask; C on the host, S x (nin nout).  PLO: into store slots from out.
    template <bool PLO>
    int combine_to(void *out, uint64_t ldo, int nin, int nout, const std::vector<double> &C,
                   const std::vector<int> &mask) {
        if (B.nchunks == 0) return QS3_OK;
        if (nout > MAXOUT) return set_err(QS3_ERR_INVALID_ARG, "at most %d vectors per combination", MAXOUT);
        const int ldc = nin * nout;
        DevBuf dC, dm;
        QS3_TRY(dC.alloc(C.size() * 8));
        QS3_TRY(dm.alloc(mask.size() * 4));
        QS3_CUDA(cudaMemcpyAsync(dC.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, st));
        QS3_CUDA(cudaMemcpyAsync(dm.p, mask.data(), mask.size() * 4, cudaMemcpyHostToDevice, st));
        k_comb64<VT, PLO><<<grid(), NTHREADS, ldc * sizeof(double), st>>>(out, ldo, V.as<ST>(), D, nin, nout,
                                                                          dC.as<double>(), ldc, secs(), c0(), B.S,
                                                                          dm.as<int>());
        QS3_LAUNCHED();
        QS3_CUDA(cudaStreamSynchronize(st));     // dC/dm are released on return
        return QS3_OK;
    }
    template <typename OT>
    int combine(OT *out, uint64_t ldo, int nin, int nout, const std::vector<double> &C, const std::vector<int> &mask) {
        static_assert(std::is_same<OT, WT>::value, "results are binary64 vectors");
        return combine_to<false>(out, ldo, nin, nout, C, mask);
    }
    // the digit store of slots j0 .. j0 + n - 1 from the binary64 store
    int digitize(int j0, int n) {
        if (B.nchunks == 0 || n <= 0) return QS3_OK;
        k_digitize<VT><<<dim3(B.nchunks, n), XT, 0, st>>>(V.as<ST>(), D, j0, DG.as<typename DigT<VT>::T>(),
                                                           GE.as<int>(), B.nchunks, secs(), c0(), B.S);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    // thick restart (Alg. 10 lines 14-19): psi_y = Psi C[:, y] for y < NK
    // (through the scratch slots), psi_NK = psi_NM; hin already holds psi_NM
    int thick_restart(int NM, int NK, const std::vector<double> &C) {
        QS3_TRY(combine_to<true>(svec(cap), 0, NM, NK, C, h_active));
        QS3_CUDA(cudaMemcpyAsync(svec(0), svec(cap), (size_t)NK * slot_bytes(), cudaMemcpyDeviceToDevice, st));
        QS3_CUDA(cudaMemcpyAsync(svec(NK), svec(NM), slot_bytes(), cudaMemcpyDeviceToDevice, st));
        return digitize(0, NK + 1);
    }
};

}  // namespace qs3
