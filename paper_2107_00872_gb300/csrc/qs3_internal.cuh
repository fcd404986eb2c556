// qs3_internal.cuh -- host structures and device helpers shared by the
// libqs3 translation units (GPU path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qs3.h"

namespace qs3 {

constexpr int MAXND = QS3_MAX_NDOWN;
constexpr int TILE = 256;          // rows per tile (one thread per row)
constexpr int NTHREADS = 256;
constexpr int BROWS = 2048;        // rows per chunk of the vector kernels (8 per thread)
// every kernel with dynamic shared memory gets this one limit (bases larger
// than it are rejected at creation), so concurrent host threads setting the
// attribute never disagree
constexpr int MAX_DYN_SMEM = 200 * 1024;

// ------------------------------------------------------------------ errors
int set_err(int code, const char *fmt, ...);
void clear_err();
const char *last_err();

#define QS3_CUDA(call)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return ::qs3::set_err(e_ == cudaErrorMemoryAllocation ? QS3_ERR_OOM : QS3_ERR_CUDA,   \
                                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,       \
                                  __LINE__);                                                       \
    } while (0)

// every kernel launch of the library is followed by QS3_LAUNCHED(): it counts
// the launch (qs3_kernel_launches) and turns a launch error into a status
void count_launch(long long n = 1);   // n < 0 takes back launches that were only captured
#define QS3_LAUNCHED()                                                                             \
    do {                                                                                           \
        ::qs3::count_launch();                                                                     \
        QS3_CUDA(cudaGetLastError());                                                              \
    } while (0)

#define QS3_TRY(expr)                                                                              \
    do {                                                                                           \
        int s_ = (expr);                                                                           \
        if (s_ != QS3_OK) return s_;                                                               \
    } while (0)

// owning device buffer
struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void release();
    int alloc(size_t bytes);                      // cudaMalloc, QS3_ERR_OOM on failure
    int upload(const void *src, size_t bytes);    // alloc + H2D copy
    template <class T> T *as() const { return (T *)p; }
};

// ------------------------------------------------------- device-side views

// Lattice data needed by every kernel.  binom rows m = 0..nd+2, each of
// np1 = N + 1 entries: binom[m * np1 + c] = C(c, m).
struct LatView {
    int N, nd, np1;
    int L[3];
    int has_k;
    int key_bits;                 // bits per site of a packed key, 0 -> compare ranks
    const uint64_t *binom;
    const int *adj_ptr;           // N + 1
    const int *adj_nbr;           // 2 n_bonds
    const double *adj_jxy;        // 2 n_bonds: hop amplitude J^xy / 2 of the bond
    const double *adj_jz;         // 2 n_bonds
    const float *adj_jxy_f;       // fp32 copy of adj_jxy
    const double *u;              // N: -(1/2) sum_j Jz_ij + h_i
    double c0;                    // sum_b Jz_b / 4 - (1/2) sum_i h_i
    const float *u_f;             // fp32 copies of u, c0 and adj_jz for the fp32 kernels
    float c0f;
    const float *adj_jz_f;
    // the fp32 remainders v - fl32(v) of adj_jxy, u, adj_jz and c0: with the
    // fp32 copies they are the double-float constants of the C128DF product
    const float *adj_jxy_lo;
    const float *u_lo;
    const float *adj_jz_lo;
    float c0lo;
    const uint32_t *xyz;          // N: the site's cell coordinates x | y << 11 | z << 22
    int nsub;                     // spins per unit cell: site r is spin r % nsub of cell r / nsub
    int ncell;                    // cells, the order of the translation group
    // representative table (k-sectors, optional): for every state a, by its
    // rank0, orb[rank0] = g << 12 | u, where the orbit's representative is the
    // g-th of the sorted list of all representatives and a = T_u (rep): the
    // translation by -u (u the flat site index) takes a to its representative
    const uint32_t *orb;
    uint32_t n_orb;               // orbits in the table (entries >= n_orb << 12 are invalid)
    double jh_uniform;            // the hop amplitude J^xy / 2 when every bond has the same one, else 0
    // fixed-width adjacency (largest degree <= 6): pad_w entries per site,
    // (neighbour, fp32 hop amplitude bits) and fp32 J^z; a site with fewer
    // neighbours is padded with itself and zero couplings
    const int2 *adj_pad;
    const float *adj_jz_pad;
    int pad_w;                    // 4 or 6; 0 when the table is not built
};

struct SecView {
    const uint64_t *sigma;        // sorted rank0 of the representatives (NULL: U(1))
    const uint8_t *stab;          // |Stab| of each representative
    const uint32_t *pidx;         // prefix index over sigma (see build_pidx)
    uint64_t dim;
    uint64_t off;                 // offset of the sector in a concatenated vector
    int K[3];
    int tile0;                    // first tile of the sector
    const double2 *ph64;          // k-sectors: per-site phases e^{-2 pi i K.r/L} (fp64) ...
    const float2 *ph32;           // ... and their fp32 copy; NULL for U(1)
    const float4 *phdf;           // ... and their double-float split (re.hi, re.lo, im.hi, im.lo)
    const int32_t *t2;            // with the representative table: orbit g -> row of this sector, -1 if absent
};

// ---------------------------------------------------------- host basis
struct Basis {
    int N = 0, nd = 0, nb = 0;
    int L[3] = {0, 0, 0};
    int nsub = 1, ncell = 0;                // spins per cell, cells (the group order)
    bool has_k = false;
    int S = 0;                              // sectors
    std::vector<int> K;                     // 3 S
    std::vector<uint64_t> dims, offs;       // S, S + 1
    uint64_t total = 0;
    std::vector<int> tile0;                 // S + 1
    int ntiles = 0;
    std::vector<int> chunk0;                // S + 1, chunks of BROWS rows (vector kernels)
    int nchunks = 0;
    // host copies of the model
    std::vector<int> bi, bj;
    std::vector<double> jxy, jz, h, pos;
    bool has_h = false;
    // device data
    DevBuf d_binom, d_adj_ptr, d_adj_nbr, d_adj_jxy, d_adj_jz, d_adj_jxy_f, d_u, d_xyz;
    DevBuf d_u_f, d_adj_jz_f;
    DevBuf d_adj_jxy_lo, d_u_lo, d_adj_jz_lo;
    DevBuf d_adj_pad, d_adj_jz_pad;         // fixed-width adjacency (LatView::adj_pad)
    std::vector<DevBuf> d_sigma, d_stab, d_pidx;
    DevBuf d_ph64, d_ph32, d_phdf;          // S x N per-site phase tables (k-sectors)
    DevBuf d_secs, d_tile0, d_chunk0;
    LatView lv{};
    std::vector<SecView> secs;
    uint64_t nnz = 0;                       // structural non-zeros (count_nnz), total and per sector
    std::vector<uint64_t> nnz_sec;
    bool nnz_valid = false;
    size_t smem_bytes = 0;                  // dynamic shared memory of the row kernels
    DevBuf d_orb, d_t2;                     // representative table (LatView::orb, SecView::t2)
    uint64_t n_orb = 0;                     // orbits (all representatives) when the table exists
    DevBuf d_oreps, d_ostab;                // with the table: each orbit's representative (rank0) and |Stab|
    DevBuf d_phdig;                         // with the table: S x N phases as digits on 2^-52 (int4)
    // autotuned launch choices, 0 = not yet tuned: resident H Phi blocks per
    // SM per vector dtype (the persistent grid, i.e. rows in flight per SM),
    // and basis vectors per pass of the double-float dot products
    int tune_hphi[5] = {0, 0, 0, 0, 0};     // indexed by qs3_dtype
    int tune_hphix = 0;                     // the same for the binary64 engine's integer H Phi
    int tune_nv = 0;
    int tune_nv64 = 0;                      // the same for the binary64 dot products (IEEE engine)
    bool narrow_ranks = false;              // U(1) with C(N, N_down) < 2^32: 32-bit rank kernels apply
    // stored terms of the k-sector H Phi (opt-in): row pointers, target rows,
    // codes (u | st << 12 | q << 16) and per-row diagonals
    DevBuf d_trp, d_tcol, d_tcode, d_tdiag;
    uint64_t n_terms = 0;
    bool stored_terms = false;
    int max_degree = 0;                     // largest number of adjacency entries of a site
};

// sector of tile t (binary search over tile0[0..S])
__device__ __forceinline__ int sector_of_tile(const int *tile0, int S, int t) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// --------------------------------------------------- combinatorial helpers

// ascending bubble network on registers (static indexing only)
template <int ND>
__device__ __forceinline__ void sort_net(int (&a)[ND]) {
#pragma unroll
    for (int i = 0; i < ND; ++i) {
#pragma unroll
        for (int j = 0; j < ND - 1 - i; ++j) {
            int lo = min(a[j], a[j + 1]);
            int hi = max(a[j], a[j + 1]);
            a[j] = lo;
            a[j + 1] = hi;
        }
    }
}

// rank0 = sum_m C(c_m, m + 1) of an ascending list (Eq. a_of_n, 0-based)
template <int ND>
__device__ __forceinline__ uint64_t rank_of(const int (&c)[ND], const uint64_t *__restrict__ sC, int np1) {
    uint64_t r = 0;
#pragma unroll
    for (int m = 0; m < ND; ++m) r += sC[(m + 1) * np1 + c[m]];
    return r;
}

// largest x in [m-1, hi] with C(x, m) <= r (col = column m of the table).
// C(x, m) ~ (x - (m-1)/2)^m / m! gives a float estimate of x; the exact table
// values then correct it by a step or two, with a binary search as fallback,
// so the result is exact for every r.
__device__ __forceinline__ int col_search(const uint64_t *__restrict__ col, int m, int hi, uint64_t r) {
    // log2(m!) for m = 0..8
    constexpr float lf[9] = {0.f, 0.f, 1.f, 2.5849625f, 4.5849625f, 6.9068906f, 9.4918531f, 12.299208f, 15.299208f};
    int x = m - 1;
    if (r > 0) {
        // uint64 -> float through two 32-bit halves (a 64-bit conversion would use the fp64 unit)
        const float rf = (float)(uint32_t)(r >> 32) * 4294967296.f + (float)(uint32_t)r;
        const float e = exp2f((__log2f(rf) + lf[m]) / (float)m) + 0.5f * (float)(m - 1);
        x = (int)e;
    }
    x = max(m - 1, min(x, hi));
#pragma unroll 1
    for (int it = 0; it < 3 && x < hi && col[x + 1] <= r; ++it) ++x;
#pragma unroll 1
    for (int it = 0; it < 3 && col[x] > r; ++it) --x;
    if (col[x] > r || (x < hi && col[x + 1] <= r)) {
        int lo = m - 1, h = hi;
        while (lo < h) {
            const int mid = (lo + h + 1) >> 1;
            if (col[mid] <= r) lo = mid; else h = mid - 1;
        }
        x = lo;
    }
    return x;
}

// inverse of rank_of (Alg. 1): greedy largest-first column search
template <int ND>
__device__ __forceinline__ void unrank(uint64_t r, const uint64_t *__restrict__ sC, int np1, int (&c)[ND]) {
    int hi = np1 - 2;
#pragma unroll
    for (int m = ND; m >= 2; --m) {
        const uint64_t *col = sC + m * np1;
        const int x = col_search(col, m, hi, r);
        c[m - 1] = x;
        r -= col[x];
        hi = x - 1;
    }
    if (ND >= 1) c[0] = (int)r;
}

// 32-bit forms for state spaces with C(N, N_down) < 2^32: every binomial a
// rank needs (rows 0..N_down) then fits 32 bits
template <int ND>
__device__ __forceinline__ uint32_t rank_of32(const int (&c)[ND], const uint32_t *__restrict__ sC, int np1) {
    uint32_t r = 0;
#pragma unroll
    for (int m = 0; m < ND; ++m) r += sC[(m + 1) * np1 + c[m]];
    return r;
}

__device__ __forceinline__ int col_search32(const uint32_t *__restrict__ col, int m, int hi, uint32_t r) {
    constexpr float lf[9] = {0.f, 0.f, 1.f, 2.5849625f, 4.5849625f, 6.9068906f, 9.4918531f, 12.299208f, 15.299208f};
    int x = m - 1;
    if (r > 0) x = (int)(exp2f((__log2f((float)r) + lf[m]) / (float)m) + 0.5f * (float)(m - 1));
    x = max(m - 1, min(x, hi));
#pragma unroll 1
    for (int it = 0; it < 3 && x < hi && col[x + 1] <= r; ++it) ++x;
#pragma unroll 1
    for (int it = 0; it < 3 && col[x] > r; ++it) --x;
    if (col[x] > r || (x < hi && col[x + 1] <= r)) {
        int lo = m - 1, h = hi;
        while (lo < h) {
            const int mid = (lo + h + 1) >> 1;
            if (col[mid] <= r) lo = mid; else h = mid - 1;
        }
        x = lo;
    }
    return x;
}

template <int ND>
__device__ __forceinline__ void unrank32(uint32_t r, const uint32_t *__restrict__ sC, int np1, int (&c)[ND]) {
    int hi = np1 - 2;
#pragma unroll
    for (int m = ND; m >= 2; --m) {
        const uint32_t *col = sC + m * np1;
        const int x = col_search32(col, m, hi, r);
        c[m - 1] = x;
        r -= col[x];
        hi = x - 1;
    }
    if (ND >= 1) c[0] = (int)r;
}

// select a[i] for a runtime i without dynamic register indexing
template <int ND>
__device__ __forceinline__ int pick(const int (&a)[ND], int i) {
    int v = a[0];
#pragma unroll
    for (int m = 1; m < ND; ++m) v = (i == m) ? a[m] : v;
    return v;
}

template <int ND>
__device__ __forceinline__ bool seen_before(const int (&a)[ND], int i, int v) {
    bool s = false;
#pragma unroll
    for (int m = 0; m < ND - 1; ++m) s |= (m < i) && (a[m] == v);
    return s;
}

// Minimum-rank translate of the site list t (the representative of its
// orbit, Alg. 7), found without trying every translation.  Translations move
// unit cells; a site is spin sb of cell (x, y, z), index sb + nsub (x + Lx
// (y + Ly z)), so the order of sites follows their cells first.
//
// The rank order is the lexicographic order of the descending list of site
// indices r = x + Lx (y + Ly z), so a representative first minimises its
// largest site, which is the (z, y, x)-largest spin.  Hence, exactly:
//  - a representative has a spin at x = 0, one at y = 0 and one at z = 0
//    (otherwise a -1 shift along that axis lowers every site index), so the
//    shifts along each axis are taken from the spins' coordinates;
//  - level z: keep the z-shifts that minimise max z' over all spins;
//  - level y: for those, keep the y-shifts that minimise max y' over the
//    spins at the top z';
//  - level x: likewise max x' over the spins at the top (z', y').
// Every surviving translation gives the same largest site; the full keys
// (sorted lists) of the survivors -- usually one -- decide.  On return rep
// holds the sorted representative, (ax, by, cz) the coordinates moved to the
// origin (T^t a' = rep with t = -(ax, by, cz)), and the function returns its
// rank0.
template <int ND>
__device__ __forceinline__ uint64_t canon(const int (&t)[ND], const LatView &L, const uint32_t *__restrict__ sxyz,
                                          const uint64_t *__restrict__ sC, int (&rep)[ND], int &ax, int &by,
                                          int &cz) {
    int X[ND], Y[ND], Z[ND], SB[ND];
#pragma unroll
    for (int m = 0; m < ND; ++m) {
        uint32_t p = sxyz[t[m]];
        X[m] = p & 2047u;
        Y[m] = (p >> 11) & 2047u;
        Z[m] = p >> 22;
        SB[m] = L.nsub > 1 ? t[m] % L.nsub : 0;     // the spin's place in its cell
    }
    const int Lx = L.L[0], Ly = L.L[1], Lz = L.L[2];
    const int kb = L.key_bits;
    // level z
    uint32_t mz = 1u;
    int bz = 0;
    if (Lz > 1) {
        bz = 0x7fffffff;
        mz = 0u;
#pragma unroll
        for (int c = 0; c < ND; ++c) {
            bool dup = false;
#pragma unroll
            for (int k = 0; k < c; ++k) dup |= (Z[k] == Z[c]);
            int mx = 0;
#pragma unroll
            for (int m = 0; m < ND; ++m) {
                int d = Z[m] - Z[c];
                d += (d < 0) ? Lz : 0;
                mx = max(mx, d);
            }
            if (!dup) {
                if (mx < bz) { bz = mx; mz = 1u << c; }
                else if (mx == bz) mz |= 1u << c;
            }
        }
    }
    uint64_t best = ~0ull;
    int bc = 0, bb = 0, ba = 0;
    for (uint32_t m1 = mz; m1; m1 &= m1 - 1) {
        const int c = __ffs(m1) - 1;
        const int zc = pick(Z, c);
        int zz[ND];
        uint32_t tz = 0u;
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            int d = Z[m] - zc;
            d += (d < 0) ? Lz : 0;
            zz[m] = d;
            tz |= (d == bz ? 1u : 0u) << m;
        }
        // level y over the top-z spins
        uint32_t my = 1u;
        int byv = 0;
        if (Ly > 1) {
            byv = 0x7fffffff;
            my = 0u;
#pragma unroll
            for (int b = 0; b < ND; ++b) {
                bool dup = false;
#pragma unroll
                for (int k = 0; k < b; ++k) dup |= (Y[k] == Y[b]);
                int mx = -1;
#pragma unroll
                for (int m = 0; m < ND; ++m) {
                    int d = Y[m] - Y[b];
                    d += (d < 0) ? Ly : 0;
                    mx = ((tz >> m) & 1u) ? max(mx, d) : mx;
                }
                if (!dup) {
                    if (mx < byv) { byv = mx; my = 1u << b; }
                    else if (mx == byv) my |= 1u << b;
                }
            }
        }
        for (uint32_t m2 = my; m2; m2 &= m2 - 1) {
            const int b = __ffs(m2) - 1;
            const int yb = pick(Y, b);
            int yy[ND];
            uint32_t ty = 0u;
#pragma unroll
            for (int m = 0; m < ND; ++m) {
                int d = Y[m] - yb;
                d += (d < 0) ? Ly : 0;
                yy[m] = d;
                ty |= (((tz >> m) & 1u) && d == byv ? 1u : 0u) << m;
            }
            // level x over the top-(z, y) spins
            uint32_t mx3 = 1u;
            if (Lx > 1) {
                int bxv = 0x7fffffff;
                mx3 = 0u;
#pragma unroll
                for (int a = 0; a < ND; ++a) {
                    bool dup = false;
#pragma unroll
                    for (int k = 0; k < a; ++k) dup |= (X[k] == X[a]);
                    int mx = -1;
#pragma unroll
                    for (int m = 0; m < ND; ++m) {
                        int d = X[m] - X[a];
                        d += (d < 0) ? Lx : 0;
                        mx = ((ty >> m) & 1u) ? max(mx, d) : mx;
                    }
                    if (!dup) {
                        if (mx < bxv) { bxv = mx; mx3 = 1u << a; }
                        else if (mx == bxv) mx3 |= 1u << a;
                    }
                }
            }
            for (uint32_t m3 = mx3; m3; m3 &= m3 - 1) {
                const int a = __ffs(m3) - 1;
                const int xa = pick(X, a);
                int s[ND];
#pragma unroll
                for (int m = 0; m < ND; ++m) {
                    int d = X[m] - xa;
                    d += (d < 0) ? Lx : 0;
                    s[m] = SB[m] + L.nsub * (d + Lx * (yy[m] + Ly * zz[m]));
                }
                sort_net(s);
                uint64_t key;
                if (kb) {
                    key = 0;
#pragma unroll
                    for (int m = ND - 1; m >= 0; --m) key = (key << kb) | (uint64_t)s[m];
                } else {
                    key = rank_of(s, sC, L.np1);
                }
                if (key < best) {
                    best = key;
                    bc = c; bb = b; ba = a;
#pragma unroll
                    for (int m = 0; m < ND; ++m) rep[m] = s[m];
                }
            }
        }
    }
    ax = pick(X, ba);
    by = pick(Y, bb);
    cz = pick(Z, bc);
    return kb ? rank_of(rep, sC, L.np1) : best;
}

// prefix of a sorted list used by the two-level index over sigma: the colex
// rank of its two largest sites (its largest site when ND == 1)
template <int ND>
__device__ __forceinline__ uint32_t prefix_of(const int (&c)[ND], const uint64_t *__restrict__ sC, int np1) {
    if (ND >= 2) return (uint32_t)(sC[2 * np1 + c[ND - 1]] + (uint64_t)c[ND - 2]);
    return (uint32_t)c[0];
}

// position of rank r in sector sv (binary search inside the prefix bucket)
__device__ __forceinline__ bool sigma_find(const SecView &sv, uint32_t P, uint64_t r, uint32_t &idx) {
    uint32_t lo = __ldg(sv.pidx + P), hi = __ldg(sv.pidx + P + 1);
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(sv.sigma + mid) < r) lo = mid + 1; else hi = mid;
    }
    idx = lo;
    return lo < __ldg(sv.pidx + P + 1) && __ldg(sv.sigma + lo) == r;
}

// stage the binomial table (rows 0..nd+2) and the coordinate table in smem
__device__ __forceinline__ void stage_tables(const LatView &L, uint64_t *sC, uint32_t *sxyz) {
    const int nC = (L.nd + 3) * L.np1;
    for (int i = threadIdx.x; i < nC; i += blockDim.x) sC[i] = L.binom[i];
    if (sxyz)
        for (int i = threadIdx.x; i < L.N; i += blockDim.x) sxyz[i] = L.xyz[i];
}

size_t row_kernel_smem(const Basis &B, int extra_nd);

// -------------------------------------------------------------- entry points
// implemented in qs3_hphi.cu
int hphi_launch(Basis &B, qs3_dtype dt, const void *phi, void *psi, cudaStream_t st,
                const int *active = nullptr);
// C128DF product: phi in double-float form (float4 per element), or phi +
// (*dx) ld when dx (device) is given; psi complex128, or double-float when out_df
int hphi_df_launch(Basis &B, const void *phi, const int *dx, uint64_t ld, void *psi, cudaStream_t st,
                   const int *active = nullptr, bool out_df = false);
int count_nnz(Basis &B, uint64_t *nnz);
// the binary64 engine's H Phi on the integer units (qs3_hphi.cu, k_hphi_x and the
// orbit-batched k_hphi_o): phi as binary64 and as its digit-store image (dg, ge:
// slot *dx of the store when dx is given)
bool hphi_x_ok(const Basis &B);
int hphi_x_launch(Basis &B, const void *phi, const void *dg, const int *ge, const int *dx, void *psi, cudaStream_t st,
                  const int *active = nullptr);
// qs3_hphi with QS3_C128X: phi's digit image in scratch, then hphi_x_launch
// (qs3_solver.cu, where the digit kernels live); synchronous on st
int hphi_x_binary64(Basis &B, const void *phi, void *psi, cudaStream_t st);
// representative table: build (QS3_OK, or an error when it cannot be built) / release
int build_rep_table(Basis &B, size_t max_bytes);
// stored-term H Phi of k-sector bases: build (QS3_OK or an error) / release / apply
int build_terms(Basis &B, size_t max_bytes);
void drop_terms(Basis &B);
int hphi_stored_launch(Basis &B, qs3_dtype dt, const void *phi, void *psi, cudaStream_t st, const int *active);
constexpr size_t REP_TABLE_AUTO_BYTES = (size_t)1 << 30;   // built at basis creation up to this size
void drop_rep_table(Basis &B);
// implemented in qs3_basis.cu
int build_sector_reps(Basis &B, int s);
// implemented in qs3_obs.cu
int sq_launch(int op, Basis &src, int s_src, const void *phi, Basis &dst, int s_dst, const int *Q, void *psi,
              cudaStream_t st);
int smq_launch(Basis &src, int s_src, const void *phi, Basis &dst, int s_dst, const int *Q, void *psi,
               cudaStream_t st);

}  // namespace qs3

struct qs3_basis_s {
    qs3::Basis B;
};
