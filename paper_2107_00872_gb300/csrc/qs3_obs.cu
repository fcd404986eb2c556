// qs3_obs.cu -- observables (Sec. "Calculating expectation values",
// "Multiplying an operator to state vectors ...", "Continued fraction
// expansion based on the Lanczos algorithm"): two-point functions, static
// S(q), S^-_q phi (Alg. 11) and the continued-fraction S^-(q, omega) of
// Eq. (cfe).
//
// Two-point functions.  U(1)-only bases: site-resolved.  The occupation
// matrix G_ij = sum_a |phi_a|^2 n_i(a) n_j(a) gives <s^z_i s^z_j> =
// 1/4 - (G_ii + G_jj)/2 + G_ij, and <s^+_i s^-_j> (i != j) moves the down
// spin i -> j: sum over a of conj(phi(a - i + j)) phi(a).  k-sectors: the
// translation-symmetrised operators (1/N) sum_r O(r, r + delta) are diagonal
// (zz) or hop-like (+-) in the symmetry-adapted basis, so every displacement
// delta is accumulated in one pass: P(delta) = sum |phi|^2 #{pairs at delta}
// and the hop sum of (1/N) sum_r s^+_r s^-_{r+delta}, whose pull form is the
// H Phi machinery with a "bond" of displacement -delta.
//
// S^-_q phi in pull form (derived from Alg. 11): for a row b of the target
// sector (N_down + 1, k + q), psi'_b = N^{-1/2} sum_{s in b}
// sqrt(|Stab a| / |Stab b|) e^{ik.u} e^{-iq.R_s} phi_a, with a the
// representative of b \ {s} and T^u (b \ {s}) = a (skipped when a is not in
// the source sector).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include <mutex>

#include "qs3_internal.cuh"

namespace qs3 {

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// per-axis phase tables: tab[alpha-offset + v] = exp(-2 pi i K_alpha v / L_alpha)
__device__ __forceinline__ void fill_axis_phases(const int *L, const int *K, double2 *tab) {
    const int tot = L[0] + L[1] + L[2];
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        int a = (i < L[0]) ? 0 : (i < L[0] + L[1] ? 1 : 2);
        int v = i - (a == 0 ? 0 : (a == 1 ? L[0] : L[0] + L[1]));
        long long num = (long long)K[a] * v % L[a];
        double sn, cs;
        sincospi(-2.0 * (double)num / (double)L[a], &sn, &cs);
        tab[i] = make_double2(cs, sn);
    }
}

struct ObsSmem {
    uint64_t *sC;
    uint32_t *sxyz;
    double2 *phk;    // e^{-2 pi i K_alpha v / L_alpha}
    double2 *phq;    // e^{-2 pi i Q_alpha v / L_alpha}
    double *snorm;   // [0..8] sqrt(s), [9..17] 1/sqrt(s)
    double2 *hist;   // per-block histogram (N entries) or NULL
};

__host__ __device__ inline size_t obs_smem_bytes(int nd_rows, int N, const int *L, bool hist) {
    size_t s = (size_t)nd_rows * (N + 1) * 8 + (size_t)N * 4;
    s = (s + 15) & ~(size_t)15;
    s += 2 * (size_t)(L[0] + L[1] + L[2]) * 16 + 18 * 8;
    s = (s + 15) & ~(size_t)15;
    if (hist) s += (size_t)N * 16;
    return s;
}

__device__ __forceinline__ ObsSmem obs_carve(const LatView &L, unsigned char *smem, bool hist) {
    ObsSmem o;
    const int rows = L.nd + 3;
    o.sC = (uint64_t *)smem;
    o.sxyz = (uint32_t *)(o.sC + (size_t)rows * L.np1);
    size_t off = (size_t)rows * L.np1 * 8 + (size_t)L.N * 4;
    off = (off + 15) & ~(size_t)15;
    o.phk = (double2 *)(smem + off);
    o.phq = o.phk + (L.L[0] + L.L[1] + L.L[2]);
    o.snorm = (double *)(o.phq + (L.L[0] + L.L[1] + L.L[2]));
    off += 2 * (size_t)(L.L[0] + L.L[1] + L.L[2]) * 16 + 18 * 8;
    off = (off + 15) & ~(size_t)15;
    o.hist = hist ? (double2 *)(smem + off) : nullptr;
    const int nC = rows * L.np1;
    for (int i = threadIdx.x; i < nC; i += blockDim.x) o.sC[i] = L.binom[i];
    for (int i = threadIdx.x; i < L.N; i += blockDim.x) o.sxyz[i] = L.xyz[i];
    if (threadIdx.x < 9) {
        o.snorm[threadIdx.x] = sqrt((double)threadIdx.x);
        o.snorm[9 + threadIdx.x] = threadIdx.x ? 1.0 / sqrt((double)threadIdx.x) : 0.0;
    }
    if (hist)
        for (int i = threadIdx.x; i < L.N; i += blockDim.x) o.hist[i] = make_double2(0.0, 0.0);
    return o;
}

__device__ __forceinline__ int disp_index(uint32_t pa, uint32_t pb, const int *L) {
    int dx = (int)(pb & 2047u) - (int)(pa & 2047u);
    int dy = (int)((pb >> 11) & 2047u) - (int)((pa >> 11) & 2047u);
    int dz = (int)(pb >> 22) - (int)(pa >> 22);
    dx += dx < 0 ? L[0] : 0;
    dy += dy < 0 ? L[1] : 0;
    dz += dz < 0 ? L[2] : 0;
    return dx + L[0] * (dy + L[1] * dz);
}

// ---------------------------------------------------------------- U(1): zz
// G[i*N + j] += |phi_a|^2 for every ordered pair of down spins (i, j) of a
// (diag_only: only i == j); norm[0] += |phi_a|^2
template <int ND, typename VT>
__global__ void __launch_bounds__(NTHREADS) k_occ_u1(LatView L, uint64_t dim, const VT *__restrict__ phi,
                                                     int diag_only, double *__restrict__ G, double *__restrict__ norm) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sC = (uint64_t *)smem;
    double *sh = (double *)(sC + (size_t)(L.nd + 3) * L.np1);
    const int nC = (L.nd + 3) * L.np1;
    for (int i = threadIdx.x; i < nC; i += blockDim.x) sC[i] = L.binom[i];
    for (int i = threadIdx.x; i <= L.N; i += blockDim.x) sh[i] = 0.0;
    __syncthreads();
    for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < dim;
         row += (uint64_t)gridDim.x * blockDim.x) {
        const VT v = phi[row];
        double w;
        if constexpr (sizeof(VT) == 16) w = ((const double2 &)v).x * ((const double2 &)v).x + ((const double2 &)v).y * ((const double2 &)v).y;
        else w = (double)(*(const double *)&v) * (double)(*(const double *)&v);
        int c[ND];
        unrank(row, sC, L.np1, c);
        atomicAdd(sh + L.N, w);
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            atomicAdd(sh + c[m], w);
            if (!diag_only)
#pragma unroll
                for (int q = 0; q < ND; ++q)
                    if (q != m) atomicAdd(G + (size_t)c[m] * L.N + c[q], w);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L.N; i += blockDim.x)
        if (sh[i] != 0.0) atomicAdd(G + (size_t)i * L.N + i, sh[i]);
    if (threadIdx.x == 0) atomicAdd(norm, sh[L.N]);
}

// --------------------------------------------------------------- U(1): +-
// M[i*N + j] += conj(phi(a - i + j)) phi(a) for i in a, j not in a
template <int ND, typename VT>
__global__ void __launch_bounds__(NTHREADS) k_spsm_u1(LatView L, uint64_t dim, const VT *__restrict__ phi,
                                                      double2 *__restrict__ M) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sC = (uint64_t *)smem;
    const int nC = (L.nd + 3) * L.np1;
    for (int i = threadIdx.x; i < nC; i += blockDim.x) sC[i] = L.binom[i];
    __syncthreads();
    for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < dim;
         row += (uint64_t)gridDim.x * blockDim.x) {
        double2 x;
        if constexpr (sizeof(VT) == 16) x = *(const double2 *)(phi + row);
        else x = make_double2(*(const double *)(phi + row), 0.0);
        int c[ND];
        unrank(row, sC, L.np1, c);
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            for (int j = 0; j < L.N; ++j) {
                bool occ = false;
#pragma unroll
                for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                if (occ) continue;
                int tt[ND];
#pragma unroll
                for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                sort_net(tt);
                const uint64_t r2 = rank_of(tt, sC, L.np1);
                double2 y;
                if constexpr (sizeof(VT) == 16) y = *(const double2 *)(phi + r2);
                else y = make_double2(*(const double *)(phi + r2), 0.0);
                // conj(y) * x
                const double re = y.x * x.x + y.y * x.y, im = y.x * x.y - y.y * x.x;
                double2 *dst = M + (size_t)c[m] * L.N + j;
                atomicAdd(&dst->x, re);
                atomicAdd(&dst->y, im);
            }
        }
    }
}

// ------------------------------------------------------------- k-sectors
// zz: hist[delta].x += |phi|^2 #{ordered pairs (m, q) at displacement delta}
// +-: hist[delta] += (1/N) conj(phi_a) (B_delta phi)_a, B_delta = sum_r s^+_r s^-_{r+delta}
template <int ND>
__global__ void __launch_bounds__(NTHREADS) k_corr_k(LatView L, SecView sv, const double2 *__restrict__ phi,
                                                     int do_pm, double2 *__restrict__ hzz, double2 *__restrict__ hpm,
                                                     double *__restrict__ norm) {
    extern __shared__ __align__(16) unsigned char smem[];
    ObsSmem sm = obs_carve(L, smem, true);
    __shared__ double snorm_acc;
    if (threadIdx.x == 0) snorm_acc = 0.0;
    fill_axis_phases(L.L, sv.K, sm.phk);
    __syncthreads();
    const double2 *phk = sm.phk;
    const double2 *phy = phk + L.L[0], *phz = phk + L.L[0] + L.L[1];
    // pass 1 (zz) uses sm.hist; pass 2 (+-) goes straight to global memory
    for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < sv.dim;
         row += (uint64_t)gridDim.x * blockDim.x) {
        const double2 x = phi[row];
        const double w = x.x * x.x + x.y * x.y;
        int c[ND];
        unrank(__ldg(sv.sigma + row), sm.sC, L.np1, c);
        atomicAdd(&snorm_acc, w);
#pragma unroll
        for (int m = 0; m < ND; ++m)
#pragma unroll
            for (int q = 0; q < ND; ++q) {
                const int d = disp_index(sm.sxyz[c[m]], sm.sxyz[c[q]], L.L);
                atomicAdd(&sm.hist[d].x, w);
            }
        if (!do_pm) continue;
        const double rs = sm.snorm[9 + __ldg(sv.stab + row)];
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            for (int j = 0; j < L.N; ++j) {
                bool occ = false;
#pragma unroll
                for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                if (occ) continue;
                int tt[ND];
#pragma unroll
                for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                sort_net(tt);
                int rep[ND];
                int ax, by, cz;
                const uint64_t r2 = canon(tt, L, sm.sxyz, sm.sC, rep, ax, by, cz);
                uint32_t idx;
                if (!sigma_find(sv, prefix_of(rep, sm.sC, L.np1), r2, idx)) continue;
                // the spin moved by -delta: delta = c_m - j
                const int d = disp_index(sm.sxyz[j], sm.sxyz[c[m]], L.L);
                const double2 p = cmul2(cmul2(phk[ax], phy[by]), phz[cz]);
                const double wn = sm.snorm[__ldg(sv.stab + idx)] * rs / (double)L.N;
                const double2 y = phi[idx];
                // conj(x) * p * wn * y
                const double2 py = cmul2(p, y);
                const double re = (x.x * py.x + x.y * py.y) * wn, im = (x.x * py.y - x.y * py.x) * wn;
                atomicAdd(&hpm[d].x, re);
                atomicAdd(&hpm[d].y, im);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L.N; i += blockDim.x)
        if (sm.hist[i].x != 0.0) atomicAdd(&hzz[i].x, sm.hist[i].x);
    if (threadIdx.x == 0) atomicAdd(norm, snorm_acc);
}

// ------------------------------------------------------------- S^-_q (K10)
// psi'_b = N^{-1/2} sum_{s in b} sqrt(|Stab a| / |Stab b|) e^{ik.u} e^{-iq.R_s} phi_a
// (pull form of Alg. 11).  ND is the target N_down; the tables staged are the
// source basis' (rows 0..ND+1), which also serve to unrank the target rows.
template <int ND, bool KS>
__global__ void __launch_bounds__(NTHREADS) k_smq(LatView Ls, SecView svs, SecView svd,
                                                  const double2 *__restrict__ phsite, double inv_sqrt_n,
                                                  const double2 *__restrict__ phi, double2 *__restrict__ psi) {
    constexpr int NS = ND - 1;
    extern __shared__ __align__(16) unsigned char smem[];
    ObsSmem sm = obs_carve(Ls, smem, false);
    if (KS) fill_axis_phases(Ls.L, svs.K, sm.phk);
    __syncthreads();
    const double2 *phk = sm.phk, *phy = sm.phk + Ls.L[0], *phz = sm.phk + Ls.L[0] + Ls.L[1];
    for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < svd.dim;
         row += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t rank = KS ? __ldg(svd.sigma + row) : row;
        int c[ND];
        unrank(rank, sm.sC, Ls.np1, c);
        const double rb = KS ? sm.snorm[9 + __ldg(svd.stab + row)] : 1.0;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            int rem[NS];
#pragma unroll
            for (int k = 0; k < NS; ++k) rem[k] = (k < m) ? c[k] : c[k + 1];
            double2 coef = phsite[c[m]];
            uint64_t idx;
            if constexpr (KS) {
                int rep[NS];
                int ax, by, cz;
                const uint64_t r2 = canon(rem, Ls, sm.sxyz, sm.sC, rep, ax, by, cz);
                uint32_t i32;
                if (!sigma_find(svs, prefix_of(rep, sm.sC, Ls.np1), r2, i32)) continue;
                idx = i32;
                coef = cmul2(coef, cmul2(cmul2(phk[ax], phy[by]), phz[cz]));
                const double w = sm.snorm[__ldg(svs.stab + idx)] * rb;
                coef.x *= w;
                coef.y *= w;
            } else {
                idx = rank_of(rem, sm.sC, Ls.np1);
            }
            acc = make_double2(acc.x + coef.x * phi[idx].x - coef.y * phi[idx].y,
                               acc.y + coef.x * phi[idx].y + coef.y * phi[idx].x);
        }
        psi[row] = make_double2(acc.x * inv_sqrt_n, acc.y * inv_sqrt_n);
    }
}

// source N_down = 0 (the vacuum, |Stab| = N, momentum 0): psi'_b = N^{-1/2} sqrt(N / |Stab b|) e^{-iq.R} phi_0
__global__ void k_smq_vac(SecView svd, int ks, int N, const double2 *__restrict__ phsite,
                          const double2 *__restrict__ phi, double2 *__restrict__ psi) {
    const uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= svd.dim) return;
    const int site = ks ? (int)svd.sigma[row] : (int)row;
    double f = 1.0 / sqrt((double)N);
    if (ks) f *= sqrt((double)N / (double)svd.stab[row]);
    const double2 p = phsite[site], x = phi[0];
    psi[row] = make_double2(f * (p.x * x.x - p.y * x.y), f * (p.x * x.y + p.y * x.x));
}

// ------------------------------------------------- S^z_q and S^+_q
// The paper applies S^+_q and S^z_q "in the same manner" as Alg. 11
// (spsmsz = 1, 3).  Pull forms, with S^alpha_q = N^{-1/2} sum_s e^{-iq.R_s}
// S^alpha_s:
//  S^z_q: N_down and the representative are kept, k -> k + q.  A row b of the
//    target sector takes psi'_b = N^{-1/2} (sum_s e^{-iq.R_s} / 2 - sum_{s in b}
//    e^{-iq.R_s}) phi_b when b is also a representative of the source sector
//    (s^z_s = 1/2 - n_s; no translation, norm ratio 1), else 0.
//  S^+_q: N_down -> N_down - 1.  A row b sums over the up sites s of b:
//    psi'_b = N^{-1/2} sum_{s not in b} sqrt(|Stab a| / |Stab b|) e^{ik.u}
//    e^{-iq.R_s} phi_a, with a the representative of b + {s} and
//    T^u (b + {s}) = a (skipped when a is not in the source sector).
template <int ND, bool KS>
__global__ void __launch_bounds__(NTHREADS) k_szq(LatView Ls, SecView svs, SecView svd,
                                                  const double2 *__restrict__ phsite, double2 half_sum,
                                                  double inv_sqrt_n, const double2 *__restrict__ phi,
                                                  double2 *__restrict__ psi) {
    extern __shared__ __align__(16) unsigned char smem[];
    ObsSmem sm = obs_carve(Ls, smem, false);
    __syncthreads();
    for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < svd.dim;
         row += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t rank = KS ? __ldg(svd.sigma + row) : row;
        int c[ND];
        unrank(rank, sm.sC, Ls.np1, c);
        uint64_t idx = row;
        if constexpr (KS) {
            uint32_t i32;
            if (!sigma_find(svs, prefix_of(c, sm.sC, Ls.np1), rank, i32)) {
                psi[row] = make_double2(0.0, 0.0);
                continue;
            }
            idx = i32;
        }
        double2 f = half_sum;
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            const double2 p = phsite[c[m]];
            f.x -= p.x;
            f.y -= p.y;
        }
        const double2 x = phi[idx];
        psi[row] = make_double2(inv_sqrt_n * (f.x * x.x - f.y * x.y), inv_sqrt_n * (f.x * x.y + f.y * x.x));
    }
}

// ND is the target N_down (>= 1); the tables staged are the source basis'
template <int ND, bool KS>
__global__ void __launch_bounds__(NTHREADS) k_spq(LatView Ls, SecView svs, SecView svd,
                                                  const double2 *__restrict__ phsite, double inv_sqrt_n,
                                                  const double2 *__restrict__ phi, double2 *__restrict__ psi) {
    constexpr int NS = ND + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    ObsSmem sm = obs_carve(Ls, smem, false);
    if (KS) fill_axis_phases(Ls.L, svs.K, sm.phk);
    __syncthreads();
    const double2 *phk = sm.phk, *phy = sm.phk + Ls.L[0], *phz = sm.phk + Ls.L[0] + Ls.L[1];
    for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < svd.dim;
         row += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t rank = KS ? __ldg(svd.sigma + row) : row;
        int c[ND];
        unrank(rank, sm.sC, Ls.np1, c);
        const double rb = KS ? sm.snorm[9 + __ldg(svd.stab + row)] : 1.0;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll 1
        for (int sidx = 0; sidx < Ls.N; ++sidx) {
            bool occ = false;
#pragma unroll
            for (int k = 0; k < ND; ++k) occ |= (c[k] == sidx);
            if (occ) continue;
            int t[NS];
#pragma unroll
            for (int k = 0; k < ND; ++k) t[k] = c[k];
            t[ND] = sidx;
            sort_net(t);
            double2 coef = phsite[sidx];
            uint64_t idx;
            if constexpr (KS) {
                int rep[NS];
                int ax, by, cz;
                const uint64_t r2 = canon(t, Ls, sm.sxyz, sm.sC, rep, ax, by, cz);
                uint32_t i32;
                if (!sigma_find(svs, prefix_of(rep, sm.sC, Ls.np1), r2, i32)) continue;
                idx = i32;
                coef = cmul2(coef, cmul2(cmul2(phk[ax], phy[by]), phz[cz]));
                const double w = sm.snorm[__ldg(svs.stab + idx)] * rb;
                coef.x *= w;
                coef.y *= w;
            } else {
                idx = rank_of(t, sm.sC, Ls.np1);
            }
            const double2 x = phi[idx];
            acc.x += coef.x * x.x - coef.y * x.y;
            acc.y += coef.x * x.y + coef.y * x.x;
        }
        psi[row] = make_double2(acc.x * inv_sqrt_n, acc.y * inv_sqrt_n);
    }
}

// S^+_q from N_down = 1 to the vacuum (one row): psi' = N^{-1/2} sum_s e^{-iq.R_s}
// [U(1): phi_s; k: e^{ik.R_s} sqrt(1/N) phi_0, the source's single representative
// being {0} with |Stab| = 1 and the vacuum's |Stab| = N]
__global__ void k_spq_vac(int N, int Lx, int Ly, int ks, int Kx, int Ky, int Kz, int Lz,
                          const double2 *__restrict__ phsite, const double2 *__restrict__ phi,
                          double2 *__restrict__ psi) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int s = 0; s < N; ++s) {
        double2 c = phsite[s];
        double2 x;
        if (ks) {
            const int x0 = s % Lx, y0 = (s / Lx) % Ly, z0 = s / (Lx * Ly);
            // e^{ik.u} with the translation moving s to the origin, as the per-axis tables
            const long long num = ((long long)Kx * x0 * (N / Lx) + (long long)Ky * y0 * (N / Ly) +
                                   (long long)Kz * z0 * (N / Lz)) % N;
            double sn, cs;
            sincospi(-2.0 * (double)num / (double)N, &sn, &cs);
            c = cmul2(c, make_double2(cs, sn));
            const double w = 1.0 / sqrt((double)N);
            c.x *= w;
            c.y *= w;
            x = phi[0];
        } else {
            x = phi[s];
        }
        acc.x += c.x * x.x - c.y * x.y;
        acc.y += c.x * x.y + c.y * x.x;
    }
    const double f = 1.0 / sqrt((double)N);
    psi[0] = make_double2(acc.x * f, acc.y * f);
}

// S(q, omega) = -(1/pi) Im[ norm2 / (z - a_0 - b_0^2 / (z - a_1 - ...)) ],
// z = omega + e0 - h + i eta, evaluated from the deepest level up (Eq. cfe)
__global__ void k_cfrac(int nq, int cap, const double *__restrict__ alpha, const double *__restrict__ beta,
                        const int *__restrict__ msz, const double *__restrict__ norm2, double e0, double h,
                        double eta, const double *__restrict__ omega, int nw, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq * nw) return;
    const int n = i / nw, w = i % nw;
    const int m = msz[n];
    if (m <= 0 || !(norm2[n] > 0.0)) { out[i] = 0.0; return; }
    const double zr = omega[w] + e0 - h, zi = eta;
    const double *a = alpha + (size_t)n * cap, *b = beta + (size_t)n * cap;
    double gr = zr - a[m - 1], gi = zi;
    for (int x = m - 2; x >= 0; --x) {
        const double den = gr * gr + gi * gi;
        const double b2 = b[x] * b[x];
        // g = z - a_x - b_x^2 / g
        gr = zr - a[x] - b2 * gr / den;
        gi = zi + b2 * gi / den;
    }
    const double den = gr * gr + gi * gi;
    // Im(norm2 / g) = -norm2 gi / |g|^2
    out[i] = norm2[n] * gi / den / M_PI;
}

// ---------------------------------------------------------------- host side

static int grid_for(uint64_t n) {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + NTHREADS - 1) / NTHREADS, (uint64_t)nsm * 8));
}

template <int ND>
static int corr_u1_nd(Basis &B, const double *phi, bool pm, double *G, double2 *M, double *nrm, cudaStream_t st) {
    const size_t sm1 = (size_t)(B.nd + 3) * (B.N + 1) * 8 + (size_t)(B.N + 1) * 8;
    QS3_CUDA(cudaFuncSetAttribute(k_occ_u1<ND, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
    const int g = grid_for(B.total);
    k_occ_u1<ND, double><<<g, NTHREADS, sm1, st>>>(B.lv, B.total, phi, 0, G, nrm);
    QS3_LAUNCHED();
    if (pm) {
        const size_t sm2 = (size_t)(B.nd + 3) * (B.N + 1) * 8;
        QS3_CUDA(cudaFuncSetAttribute(k_spsm_u1<ND, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_spsm_u1<ND, double><<<g, NTHREADS, sm2, st>>>(B.lv, B.total, phi, M);
        QS3_LAUNCHED();
    }
    return QS3_OK;
}

template <int ND>
static int corr_k_nd(Basis &B, int s, const double2 *phi, bool pm, double2 *hzz, double2 *hpm, double *nrm,
                     cudaStream_t st) {
    const size_t smem = obs_smem_bytes(B.nd + 3, B.N, B.L, true);
    if (smem > 200 * 1024) return set_err(QS3_ERR_OVERFLOW, "correlation tables need %zu bytes of shared memory", smem);
    QS3_CUDA(cudaFuncSetAttribute(k_corr_k<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
    k_corr_k<ND><<<grid_for(B.dims[s]), NTHREADS, smem, st>>>(B.lv, B.secs[s], phi, pm ? 1 : 0, hzz, hpm, nrm);
    QS3_LAUNCHED();
    return QS3_OK;
}

template <int ND>
static int smq_nd(Basis &S, int ss, Basis &Dd, int sd, const double2 *phs, const double2 *phi, double2 *psi,
                  cudaStream_t st) {
    if constexpr (ND < 2) {
        return set_err(QS3_ERR_INVALID_ARG, "internal: smq_nd<%d>", ND);
    } else {
        const size_t smem = obs_smem_bytes(S.nd + 3, S.N, S.L, false);
        if (smem > 200 * 1024) return set_err(QS3_ERR_OVERFLOW, "S^-_q tables need %zu bytes of shared memory", smem);
        const double isn = 1.0 / std::sqrt((double)S.N);
        if (S.has_k) {
            QS3_CUDA(cudaFuncSetAttribute(k_smq<ND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
            k_smq<ND, true><<<grid_for(Dd.dims[sd]), NTHREADS, smem, st>>>(S.lv, S.secs[ss], Dd.secs[sd], phs, isn,
                                                                            phi, psi);
        } else {
            QS3_CUDA(cudaFuncSetAttribute(k_smq<ND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
            k_smq<ND, false><<<grid_for(Dd.dims[sd]), NTHREADS, smem, st>>>(S.lv, S.secs[ss], Dd.secs[sd], phs, isn,
                                                                             phi, psi);
        }
        QS3_LAUNCHED();
        return QS3_OK;
    }
}

static int dispatch_smq(Basis &S, int ss, Basis &Dd, int sd, const double2 *phs, const double2 *phi, double2 *psi,
                        cudaStream_t st) {
    switch (Dd.nd) {
        case 2: return smq_nd<2>(S, ss, Dd, sd, phs, phi, psi, st);
        case 3: return smq_nd<3>(S, ss, Dd, sd, phs, phi, psi, st);
        case 4: return smq_nd<4>(S, ss, Dd, sd, phs, phi, psi, st);
        case 5: return smq_nd<5>(S, ss, Dd, sd, phs, phi, psi, st);
        case 6: return smq_nd<6>(S, ss, Dd, sd, phs, phi, psi, st);
        case 7: return smq_nd<7>(S, ss, Dd, sd, phs, phi, psi, st);
        case 8: return smq_nd<8>(S, ss, Dd, sd, phs, phi, psi, st);
        default: return set_err(QS3_ERR_INVALID_ARG, "target n_down %d", Dd.nd);
    }
}

static void site_pos(const Basis &B, int r, double *p) {
    if (!B.pos.empty()) {
        for (int a = 0; a < 3; ++a) p[a] = B.pos[3 * (size_t)r + a];
        return;
    }
    p[0] = r % B.L[0];
    p[1] = (r / B.L[0]) % B.L[1];
    p[2] = r / (B.L[0] * B.L[1]);
}

// e^{-i q.R_r} for every site, q.a_alpha = 2 pi Q_alpha / L_alpha
static std::vector<double2> site_phases(const Basis &B, const int *Q) {
    std::vector<double2> ph(B.N);
    for (int r = 0; r < B.N; ++r) {
        double p[3];
        site_pos(B, r, p);
        double t = 0.0;
        for (int a = 0; a < 3; ++a)
            if (B.L[a] > 0) t += 2.0 * M_PI * Q[a] * p[a] / B.L[a];    // no translation group: q = 0
        ph[r] = make_double2(std::cos(t), -std::sin(t));
    }
    return ph;
}

int smq_launch(Basis &S, int ss, const void *phi, Basis &Dd, int sd, const int *Q, void *psi, cudaStream_t st) {
    if (S.nsub > 1 || Dd.nsub > 1)
        return set_err(QS3_ERR_INVALID_ARG, "S^alpha_q takes one spin per unit cell");
    if (S.N != Dd.N || S.L[0] != Dd.L[0] || S.L[1] != Dd.L[1] || S.L[2] != Dd.L[2])
        return set_err(QS3_ERR_INVALID_ARG, "source and target bases are on different lattices");
    if (Dd.nd != S.nd + 1) return set_err(QS3_ERR_INVALID_ARG, "target n_down must be source n_down + 1");
    if (S.has_k != Dd.has_k) return set_err(QS3_ERR_INVALID_ARG, "both bases need momenta, or neither");
    if (ss < 0 || ss >= S.S || sd < 0 || sd >= Dd.S) return set_err(QS3_ERR_INVALID_ARG, "sector index");
    if (S.has_k)
        for (int a = 0; a < 3; ++a)
            if ((((long long)S.K[3 * ss + a] + Q[a]) % S.L[a] + S.L[a]) % S.L[a] != Dd.K[3 * sd + a])
                return set_err(QS3_ERR_SYMMETRY, "target momentum is not K + Q (axis %d)", a);
    if (Dd.dims[sd] == 0) return QS3_OK;
    std::vector<double2> ph = site_phases(S, Q);
    DevBuf dph;
    QS3_TRY(dph.upload(ph.data(), ph.size() * sizeof(double2)));
    if (S.dims[ss] == 0) {
        QS3_CUDA(cudaMemsetAsync(psi, 0, Dd.dims[sd] * 16, st));
        QS3_CUDA(cudaStreamSynchronize(st));
        return QS3_OK;
    }
    if (S.nd == 0) {
        k_smq_vac<<<(unsigned)((Dd.dims[sd] + 255) / 256), 256, 0, st>>>(Dd.secs[sd], Dd.has_k ? 1 : 0, S.N,
                                                                          dph.as<double2>(), (const double2 *)phi,
                                                                          (double2 *)psi);
        QS3_LAUNCHED();
    } else {
        QS3_TRY(dispatch_smq(S, ss, Dd, sd, dph.as<double2>(), (const double2 *)phi, (double2 *)psi, st));
    }
    QS3_CUDA(cudaStreamSynchronize(st));     // dph is released on return
    return QS3_OK;
}

template <int ND>
static int szq_nd(Basis &S, int ss, Basis &Dd, int sd, const double2 *phs, double2 half_sum, const double2 *phi,
                  double2 *psi, cudaStream_t st) {
    const size_t smem = obs_smem_bytes(S.nd + 3, S.N, S.L, false);
    if (smem > 200 * 1024) return set_err(QS3_ERR_OVERFLOW, "S^z_q tables need %zu bytes of shared memory", smem);
    const double isn = 1.0 / std::sqrt((double)S.N);
    if (S.has_k) {
        QS3_CUDA(cudaFuncSetAttribute(k_szq<ND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_szq<ND, true><<<grid_for(Dd.dims[sd]), NTHREADS, smem, st>>>(S.lv, S.secs[ss], Dd.secs[sd], phs, half_sum,
                                                                        isn, phi, psi);
    } else {
        QS3_CUDA(cudaFuncSetAttribute(k_szq<ND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_szq<ND, false><<<grid_for(Dd.dims[sd]), NTHREADS, smem, st>>>(S.lv, S.secs[ss], Dd.secs[sd], phs, half_sum,
                                                                         isn, phi, psi);
    }
    QS3_LAUNCHED();
    return QS3_OK;
}

template <int ND>
static int spq_nd(Basis &S, int ss, Basis &Dd, int sd, const double2 *phs, const double2 *phi, double2 *psi,
                  cudaStream_t st) {
    const size_t smem = obs_smem_bytes(S.nd + 3, S.N, S.L, false);
    if (smem > 200 * 1024) return set_err(QS3_ERR_OVERFLOW, "S^+_q tables need %zu bytes of shared memory", smem);
    const double isn = 1.0 / std::sqrt((double)S.N);
    if (S.has_k) {
        QS3_CUDA(cudaFuncSetAttribute(k_spq<ND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_spq<ND, true><<<grid_for(Dd.dims[sd]), NTHREADS, smem, st>>>(S.lv, S.secs[ss], Dd.secs[sd], phs, isn, phi,
                                                                        psi);
    } else {
        QS3_CUDA(cudaFuncSetAttribute(k_spq<ND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_spq<ND, false><<<grid_for(Dd.dims[sd]), NTHREADS, smem, st>>>(S.lv, S.secs[ss], Dd.secs[sd], phs, isn, phi,
                                                                         psi);
    }
    QS3_LAUNCHED();
    return QS3_OK;
}

#define QS3_ND_SWITCH(nd, CALL)                                            \
    switch (nd) {                                                          \
        case 1: return CALL(1);                                            \
        case 2: return CALL(2);                                            \
        case 3: return CALL(3);                                            \
        case 4: return CALL(4);                                            \
        case 5: return CALL(5);                                            \
        case 6: return CALL(6);                                            \
        case 7: return CALL(7);                                            \
        case 8: return CALL(8);                                            \
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", (nd)); \
    }

static int dispatch_szq(Basis &S, int ss, Basis &Dd, int sd, const double2 *phs, double2 hs, const double2 *phi,
                        double2 *psi, cudaStream_t st) {
#define QS3_SZQ(n) szq_nd<n>(S, ss, Dd, sd, phs, hs, phi, psi, st)
    QS3_ND_SWITCH(S.nd, QS3_SZQ)
#undef QS3_SZQ
}

static int dispatch_spq(Basis &S, int ss, Basis &Dd, int sd, const double2 *phs, const double2 *phi, double2 *psi,
                        cudaStream_t st) {
#define QS3_SPQ(n) spq_nd<n>(S, ss, Dd, sd, phs, phi, psi, st)
    QS3_ND_SWITCH(Dd.nd, QS3_SPQ)
#undef QS3_SPQ
}

// S^alpha_q phi (alpha by the paper's spsmsz code: 1 S^+, 2 S^-, 3 S^z) from
// sector ss of S into sector sd of Dd
int sq_launch(int op, Basis &S, int ss, const void *phi, Basis &Dd, int sd, const int *Q, void *psi,
              cudaStream_t st) {
    if (op == QS3_OP_SMINUS) return smq_launch(S, ss, phi, Dd, sd, Q, psi, st);
    if (op != QS3_OP_SPLUS && op != QS3_OP_SZ) return set_err(QS3_ERR_INVALID_ARG, "operator %d", op);
    if (S.nsub > 1 || Dd.nsub > 1)
        return set_err(QS3_ERR_INVALID_ARG, "S^alpha_q takes one spin per unit cell");

    if (S.N != Dd.N || S.L[0] != Dd.L[0] || S.L[1] != Dd.L[1] || S.L[2] != Dd.L[2])
        return set_err(QS3_ERR_INVALID_ARG, "source and target bases are on different lattices");
    const int want = op == QS3_OP_SPLUS ? S.nd - 1 : S.nd;
    if (Dd.nd != want || want < 0)
        return set_err(QS3_ERR_INVALID_ARG, "target n_down must be source n_down %s", op == QS3_OP_SPLUS ? "- 1" : "");
    if (S.has_k != Dd.has_k) return set_err(QS3_ERR_INVALID_ARG, "both bases need momenta, or neither");
    if (ss < 0 || ss >= S.S || sd < 0 || sd >= Dd.S) return set_err(QS3_ERR_INVALID_ARG, "sector index");
    if (S.has_k)
        for (int a = 0; a < 3; ++a)
            if ((((long long)S.K[3 * ss + a] + Q[a]) % S.L[a] + S.L[a]) % S.L[a] != Dd.K[3 * sd + a])
                return set_err(QS3_ERR_SYMMETRY, "target momentum is not K + Q (axis %d)", a);
    if (Dd.dims[sd] == 0) return QS3_OK;
    std::vector<double2> ph = site_phases(S, Q);
    double2 hs = make_double2(0.0, 0.0);
    for (const double2 &v : ph) { hs.x += 0.5 * v.x; hs.y += 0.5 * v.y; }
    DevBuf dph;
    QS3_TRY(dph.upload(ph.data(), ph.size() * sizeof(double2)));
    if (S.dims[ss] == 0) {
        QS3_CUDA(cudaMemsetAsync(psi, 0, Dd.dims[sd] * 16, st));
    } else if (op == QS3_OP_SZ) {
        if (S.nd == 0) {
            // the vacuum: S^z_q |0> = N^{-1/2} (sum_s e^{-iq.R_s} / 2) |0>
            const double f = 1.0 / std::sqrt((double)S.N);
            double2 x;
            QS3_CUDA(cudaMemcpyAsync(&x, phi, sizeof(double2), cudaMemcpyDeviceToHost, st));
            QS3_CUDA(cudaStreamSynchronize(st));
            const double2 y = make_double2(f * (hs.x * x.x - hs.y * x.y), f * (hs.x * x.y + hs.y * x.x));
            QS3_CUDA(cudaMemcpyAsync(psi, &y, sizeof(double2), cudaMemcpyHostToDevice, st));
        } else {
            QS3_TRY(dispatch_szq(S, ss, Dd, sd, dph.as<double2>(), hs, (const double2 *)phi, (double2 *)psi, st));
        }
    } else if (Dd.nd == 0) {
        k_spq_vac<<<1, 32, 0, st>>>(S.N, S.L[0], S.L[1], S.has_k ? 1 : 0, S.has_k ? S.K[3 * ss] : 0,
                                    S.has_k ? S.K[3 * ss + 1] : 0, S.has_k ? S.K[3 * ss + 2] : 0, S.L[2],
                                    dph.as<double2>(), (const double2 *)phi, (double2 *)psi);
        QS3_LAUNCHED();
    } else {
        QS3_TRY(dispatch_spq(S, ss, Dd, sd, dph.as<double2>(), (const double2 *)phi, (double2 *)psi, st));
    }
    QS3_CUDA(cudaStreamSynchronize(st));     // dph is released on return
    return QS3_OK;
}

static int dispatch_corr_u1(Basis &B, const double *phi, bool pm, double *G, double2 *M, double *nrm,
                            cudaStream_t st) {
    switch (B.nd) {
        case 1: return corr_u1_nd<1>(B, phi, pm, G, M, nrm, st);
        case 2: return corr_u1_nd<2>(B, phi, pm, G, M, nrm, st);
        case 3: return corr_u1_nd<3>(B, phi, pm, G, M, nrm, st);
        case 4: return corr_u1_nd<4>(B, phi, pm, G, M, nrm, st);
        case 5: return corr_u1_nd<5>(B, phi, pm, G, M, nrm, st);
        case 6: return corr_u1_nd<6>(B, phi, pm, G, M, nrm, st);
        case 7: return corr_u1_nd<7>(B, phi, pm, G, M, nrm, st);
        case 8: return corr_u1_nd<8>(B, phi, pm, G, M, nrm, st);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

static int dispatch_corr_k(Basis &B, int s, const double2 *phi, bool pm, double2 *hzz, double2 *hpm, double *nrm,
                           cudaStream_t st) {
    switch (B.nd) {
        case 1: return corr_k_nd<1>(B, s, phi, pm, hzz, hpm, nrm, st);
        case 2: return corr_k_nd<2>(B, s, phi, pm, hzz, hpm, nrm, st);
        case 3: return corr_k_nd<3>(B, s, phi, pm, hzz, hpm, nrm, st);
        case 4: return corr_k_nd<4>(B, s, phi, pm, hzz, hpm, nrm, st);
        case 5: return corr_k_nd<5>(B, s, phi, pm, hzz, hpm, nrm, st);
        case 6: return corr_k_nd<6>(B, s, phi, pm, hzz, hpm, nrm, st);
        case 7: return corr_k_nd<7>(B, s, phi, pm, hzz, hpm, nrm, st);
        case 8: return corr_k_nd<8>(B, s, phi, pm, hzz, hpm, nrm, st);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

static int correlations(Basis &B, int s, const void *gs, int npairs, const int *pairs, double *szsz, double *spsm,
                        double *szl, int nq, const double *q, double *sqz, double *sqp, cudaStream_t st) {
    const int N = B.N, nd = B.nd;
    if (B.has_k && B.nsub > 1)
        return set_err(QS3_ERR_INVALID_ARG, "translation-symmetrised correlations take one spin per unit cell");
    if (B.nsub > 1 && nq > 0 && B.pos.empty())
        return set_err(QS3_ERR_INVALID_ARG, "S(q) on a lattice with several spins per cell needs the site positions");
    const bool want_pm = (spsm && npairs > 0) || (sqp && nq > 0);
    for (int p = 0; p < npairs; ++p)
        if (pairs[2 * p] < 0 || pairs[2 * p] >= N || pairs[2 * p + 1] < 0 || pairs[2 * p + 1] >= N)
            return set_err(QS3_ERR_INVALID_ARG, "pair %d outside the lattice", p);
    // zz(i, j) and pm(i, j) as functions on site pairs
    std::vector<double> Gh, Ch;
    std::vector<double2> Mh, Ph;
    double norm2 = 0.0;
    if (B.dims[s] == 0) return set_err(QS3_ERR_INVALID_ARG, "sector %d is empty", s);
    if (!B.has_k) {
        DevBuf G, M, nr;
        QS3_TRY(G.alloc((size_t)N * N * 8));
        QS3_CUDA(cudaMemsetAsync(G.p, 0, (size_t)N * N * 8, st));
        QS3_TRY(nr.alloc(8));
        QS3_CUDA(cudaMemsetAsync(nr.p, 0, 8, st));
        QS3_TRY(M.alloc(want_pm ? (size_t)N * N * 16 : 16));
        QS3_CUDA(cudaMemsetAsync(M.p, 0, M.n, st));
        if (nd > 0) {
            QS3_TRY(dispatch_corr_u1(B, (const double *)gs, want_pm, G.as<double>(), M.as<double2>(), nr.as<double>(), st));
            QS3_CUDA(cudaMemcpyAsync(&norm2, nr.p, 8, cudaMemcpyDeviceToHost, st));
        } else {
            double v;
            QS3_CUDA(cudaMemcpyAsync(&v, gs, 8, cudaMemcpyDeviceToHost, st));
            QS3_CUDA(cudaStreamSynchronize(st));
            norm2 = v * v;
        }
        Gh.resize((size_t)N * N);
        QS3_CUDA(cudaMemcpyAsync(Gh.data(), G.p, Gh.size() * 8, cudaMemcpyDeviceToHost, st));
        if (want_pm) {
            Mh.resize((size_t)N * N);
            QS3_CUDA(cudaMemcpyAsync(Mh.data(), M.p, Mh.size() * 16, cudaMemcpyDeviceToHost, st));
        }
        QS3_CUDA(cudaStreamSynchronize(st));
    } else {
        DevBuf hzz, hpm, nr;
        QS3_TRY(hzz.alloc((size_t)N * 16));
        QS3_TRY(hpm.alloc((size_t)N * 16));
        QS3_TRY(nr.alloc(8));
        QS3_CUDA(cudaMemsetAsync(hzz.p, 0, hzz.n, st));
        QS3_CUDA(cudaMemsetAsync(hpm.p, 0, hpm.n, st));
        QS3_CUDA(cudaMemsetAsync(nr.p, 0, 8, st));
        if (nd > 0) {
            QS3_TRY(dispatch_corr_k(B, s, (const double2 *)gs, want_pm, hzz.as<double2>(), hpm.as<double2>(),
                                    nr.as<double>(), st));
            QS3_CUDA(cudaMemcpyAsync(&norm2, nr.p, 8, cudaMemcpyDeviceToHost, st));
        } else {
            double2 v;
            QS3_CUDA(cudaMemcpyAsync(&v, gs, 16, cudaMemcpyDeviceToHost, st));
            QS3_CUDA(cudaStreamSynchronize(st));
            norm2 = v.x * v.x + v.y * v.y;
        }
        Ph.resize(N);
        std::vector<double2> hz(N);
        QS3_CUDA(cudaMemcpyAsync(hz.data(), hzz.p, N * 16, cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaMemcpyAsync(Ph.data(), hpm.p, N * 16, cudaMemcpyDeviceToHost, st));
        QS3_CUDA(cudaStreamSynchronize(st));
        Ch.resize(N);
        for (int d = 0; d < N; ++d) Ch[d] = hz[d].x;
    }
    if (!(norm2 > 0.0)) return set_err(QS3_ERR_INVALID_ARG, "state has zero norm");
    auto disp = [&](int i, int j) {   // displacement index of j - i
        const int Lx = B.L[0], Ly = B.L[1], Lz = B.L[2];
        int dx = j % Lx - i % Lx, dy = (j / Lx) % Ly - (i / Lx) % Ly, dz = j / (Lx * Ly) - i / (Lx * Ly);
        dx += dx < 0 ? Lx : 0; dy += dy < 0 ? Ly : 0; dz += dz < 0 ? Lz : 0;
        return dx + Lx * (dy + Ly * dz);
    };
    auto n_i = [&](int i) { return B.has_k ? (double)nd / N : Gh[(size_t)i * N + i] / norm2; };
    auto zz = [&](int i, int j) -> double {
        if (i == j) return 0.25;
        if (B.has_k) return 0.25 - (double)nd / N + Ch[disp(i, j)] / (N * norm2);
        return 0.25 - 0.5 * (n_i(i) + n_i(j)) + Gh[(size_t)i * N + j] / norm2;
    };
    auto pm = [&](int i, int j) -> std::complex<double> {
        if (i == j) return 1.0 - n_i(i);
        if (B.has_k) { const double2 v = Ph[disp(i, j)]; return std::complex<double>(v.x, v.y) / norm2; }
        const double2 v = Mh[(size_t)i * N + j];
        return std::complex<double>(v.x, v.y) / norm2;
    };
    for (int p = 0; p < npairs; ++p) {
        const int i = pairs[2 * p], j = pairs[2 * p + 1];
        if (szsz) szsz[p] = zz(i, j);
        if (spsm) { const auto v = pm(i, j); spsm[2 * p] = v.real(); spsm[2 * p + 1] = v.imag(); }
    }
    if (szl)
        for (int i = 0; i < N; ++i) szl[i] = 0.5 - n_i(i);
    // S(q) = (1/N) sum_{r,r'} e^{iq.(R_r - R_r')} <O_r O_r'>
    std::vector<double> P((size_t)3 * N);
    for (int r = 0; r < N; ++r) site_pos(B, r, &P[3 * (size_t)r]);
    for (int n = 0; n < nq; ++n) {
        std::vector<std::complex<double>> e(N);
        for (int r = 0; r < N; ++r)
            e[r] = std::exp(std::complex<double>(0.0, q[3 * n] * P[3 * r] + q[3 * n + 1] * P[3 * r + 1] +
                                                           q[3 * n + 2] * P[3 * r + 2]));
        std::complex<double> az = 0.0, ap = 0.0;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                const std::complex<double> f = e[i] * std::conj(e[j]);
                if (sqz) az += f * zz(i, j);
                if (sqp) ap += f * pm(i, j);
            }
        if (sqz) sqz[n] = az.real() / N;
        if (sqp) sqp[n] = ap.real() / N;
    }
    return QS3_OK;
}

}  // namespace qs3

using namespace qs3;

extern "C" int qs3_correlations(qs3_basis_t b, int32_t s, const void *gs, int32_t n_pairs, const int32_t *pairs,
                                double *szsz, double *spsm, double *sz_local, int32_t n_q, const double *q,
                                double *sq_zz, double *sq_pm, void *stream) {
    clear_err();
    if (!b || !gs) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    if (s < 0 || s >= b->B.S) return set_err(QS3_ERR_INVALID_ARG, "sector %d", s);
    if (n_pairs < 0 || (n_pairs > 0 && !pairs) || n_q < 0 || (n_q > 0 && !q))
        return set_err(QS3_ERR_INVALID_ARG, "pair / wave-vector arrays");
    return correlations(b->B, s, gs, n_pairs, pairs, szsz, spsm, sz_local, n_q, q, sq_zz, sq_pm,
                        (cudaStream_t)stream);
}

extern "C" int qs3_smq(qs3_basis_t src, int32_t s_src, const void *phi, qs3_basis_t dst, int32_t s_dst,
                       const int32_t *Q, void *psi, void *stream) {
    clear_err();
    if (!src || !dst || !phi || !psi || !Q) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    return smq_launch(src->B, s_src, phi, dst->B, s_dst, Q, psi, (cudaStream_t)stream);
}

// implemented in qs3_solver.cu (uses the Lanczos engine)
namespace qs3 {
int dsf_run(int op, Basis &S, int ss, const void *gs, double e0, Basis &Dd, int nq, const int *Q, int n_iter,
            double eta, double h, int nw, const double *omega, double *s_qw, double *alpha, double *beta,
            double *norm2, cudaStream_t st);
int cfrac_launch(int nq, int cap, const double *alpha, const double *beta, const int *msz, const double *norm2,
                 double e0, double h, double eta, const double *omega, int nw, double *out, cudaStream_t st) {
    const int n = nq * nw;
    if (n == 0) return QS3_OK;
    k_cfrac<<<(n + 255) / 256, 256, 0, st>>>(nq, cap, alpha, beta, msz, norm2, e0, h, eta, omega, nw, out);
    QS3_LAUNCHED();
    return QS3_OK;
}
}  // namespace qs3

extern "C" int qs3_dsf(qs3_basis_t src, int32_t s_src, const void *gs, double e0, qs3_basis_t dst, int32_t n_q,
                       const int32_t *Q, int32_t n_iter, double eta, double h_field, int32_t n_omega,
                       const double *omega, double *s_qw, double *alpha, double *beta, double *norm2, void *stream) {
    clear_err();
    if (!src || !dst || !gs || !Q || (n_omega > 0 && !omega)) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    if (n_q < 1 || n_q != dst->B.S) return set_err(QS3_ERR_INVALID_ARG, "n_q %d must equal the target sectors %d", n_q, dst->B.S);
    if (n_iter < 1 || n_iter > 2047) return set_err(QS3_ERR_INVALID_ARG, "n_iter %d outside [1, 2047]", n_iter);
    if (!(eta > 0)) return set_err(QS3_ERR_INVALID_ARG, "eta must be positive");
    return dsf_run(QS3_OP_SMINUS, src->B, s_src, gs, e0, dst->B, n_q, Q, n_iter, eta, h_field, n_omega, omega, s_qw,
                   alpha, beta, norm2, (cudaStream_t)stream);
}

extern "C" int qs3_sq_apply(int32_t op, qs3_basis_t src, int32_t s_src, const void *phi, qs3_basis_t dst,
                            int32_t s_dst, const int32_t *Q, void *psi, void *stream) {
    clear_err();
    if (!src || !dst || !Q) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    if (s_src < 0 || s_src >= src->B.S || s_dst < 0 || s_dst >= dst->B.S)
        return set_err(QS3_ERR_INVALID_ARG, "sector index");
    // a vector of an empty sector may be NULL
    if ((!phi && src->B.dims[s_src] > 0) || (!psi && dst->B.dims[s_dst] > 0))
        return set_err(QS3_ERR_INVALID_ARG, "NULL vector");
    return sq_launch(op, src->B, s_src, phi, dst->B, s_dst, Q, psi, (cudaStream_t)stream);
}

extern "C" int qs3_dsf_op(int32_t op, int32_t subtract_trivial, qs3_basis_t src, int32_t s_src, const void *gs,
                          double e0, qs3_basis_t dst, int32_t n_q, const int32_t *Q, int32_t n_iter, double eta,
                          double h_field, int32_t n_omega, const double *omega, double *s_qw, double *alpha,
                          double *beta, double *norm2, void *stream) {
    clear_err();
    if (op != QS3_OP_SPLUS && op != QS3_OP_SMINUS && op != QS3_OP_SZ)
        return set_err(QS3_ERR_INVALID_ARG, "operator %d", op);
    if (!src || !dst || !gs || !Q || (n_omega > 0 && !omega)) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    if (n_q < 1 || n_q != dst->B.S) return set_err(QS3_ERR_INVALID_ARG, "n_q %d must equal the target sectors %d", n_q, dst->B.S);
    if (n_iter < 1 || n_iter > 2047) return set_err(QS3_ERR_INVALID_ARG, "n_iter %d outside [1, 2047]", n_iter);
    if (!(eta > 0)) return set_err(QS3_ERR_INVALID_ARG, "eta must be positive");
    QS3_TRY(dsf_run(op, src->B, s_src, gs, e0, dst->B, n_q, Q, n_iter, eta, h_field, n_omega, omega, s_qw, alpha,
                    beta, norm2, (cudaStream_t)stream));
    if (op == QS3_OP_SZ && subtract_trivial && s_qw && n_omega > 0) {
        const Basis &S = src->B;
        const double M = 0.5 * S.N - S.nd;
        for (int n = 0; n < n_q; ++n) {
            bool zero = true;
            for (int a = 0; a < 3; ++a) {
                const int La = std::max(S.L[a], 1);
                zero &= ((Q[3 * n + a] % La) + La) % La == 0;
            }
            if (!zero) continue;
            for (int w = 0; w < n_omega; ++w)
                s_qw[(size_t)n * n_omega + w] -= eta / (M_PI * (omega[w] * omega[w] + eta * eta)) * M * M / S.N;
        }
    }
    return QS3_OK;
}

// ----------------------------------------------- S^-_q without allocation
// qs3_smq allocates a small device table of the site phases e^{-i q.R_r}
// for every call.  qs3_smq_noalloc is the same product for callers that
// must not allocate device memory while they run -- for example code
// driven by an external memory pool or an allocator they cannot call into,
// or code running where a cudaMalloc would synchronise the device.  Its
// only scratch, that phase table, lives in the file-scope array below:
// NOALLOC_MAX_SITES = 2048 complex doubles (32 KB), held by every GPU that
// loads the library until the process exits.
namespace qs3 {

constexpr int NOALLOC_MAX_SITES = 2048;
static __device__ __align__(256) double2 g_smq_phase_scratch[NOALLOC_MAX_SITES];

// device address of the scratch on each device, with the CUDA context it
// was looked up in.  A call that is not being captured into a graph looks it
// up again (cheap, host side), so a context that was reset and recreated
// never sees a stale address; a captured call uses the cached address only
// when the current context is the one it came from.
static void *g_scratch_addr[256];
static void *g_scratch_ctx[256];
static std::atomic<int> g_scratch_ready[256];
static std::mutex g_scratch_mu;

typedef int (*CtxGetCurrentFn)(void **);

static int current_context(void **ctx) {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)f;
    });
    *ctx = nullptr;
    if (!fn || fn(ctx) != 0) return set_err(QS3_ERR_CUDA, "cuCtxGetCurrent unavailable");
    return QS3_OK;
}

static int noalloc_scratch(cudaStream_t st, double2 **out) {
    int dev = 0;
    QS3_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_err(QS3_ERR_INVALID_ARG, "device %d", dev);
    void *ctx = nullptr;
    QS3_TRY(current_context(&ctx));
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    QS3_CUDA(cudaStreamIsCapturing(st, &cst));
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (cst == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_smq_phase_scratch);
        if (e != cudaSuccess || !p)
            return set_err(QS3_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
        g_scratch_ready[dev].store(1, std::memory_order_release);
    } else if (!g_scratch_ready[dev].load(std::memory_order_acquire) || g_scratch_ctx[dev] != ctx) {
        return set_err(QS3_ERR_STATE, "qs3_smq_noalloc: call it once outside stream capture on this device "
                                      "(and context) before capturing it");
    }
    *out = (double2 *)g_scratch_addr[dev];
    return QS3_OK;
}

// ph[r] = e^{-i q.R_r} with R_r the coordinates of site r and
// q.a_alpha = 2 pi Q_alpha / L_alpha; the angle is reduced exactly in integers
__global__ void k_site_phases(int N, int Lx, int Ly, int Lz, int Qx, int Qy, int Qz, double2 *__restrict__ ph) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const long long x = r % Lx, y = (r / Lx) % Ly, z = r / (Lx * Ly);
    long long num = ((long long)Qx * x * (N / Lx) + (long long)Qy * y * (N / Ly) + (long long)Qz * z * (N / Lz)) % N;
    num += num < 0 ? N : 0;
    double sn, cs;
    sincospi(2.0 * (double)num / (double)N, &sn, &cs);
    ph[r] = make_double2(cs, -sn);
}

static int smq_noalloc(Basis &S, int ss, const void *phi, Basis &Dd, int sd, const int *Q, void *psi,
                       cudaStream_t st) {
    if (S.nsub > 1 || Dd.nsub > 1)
        return set_err(QS3_ERR_INVALID_ARG, "S^alpha_q takes one spin per unit cell");
    if (S.N > NOALLOC_MAX_SITES)
        return set_err(QS3_ERR_INVALID_ARG, "n_sites %d exceeds the %d sites of the no-allocation scratch", S.N,
                       NOALLOC_MAX_SITES);
    if (!S.pos.empty())
        return set_err(QS3_ERR_INVALID_ARG, "the no-allocation S^-_q takes lattices without a position array");
    if (S.N != Dd.N || S.L[0] != Dd.L[0] || S.L[1] != Dd.L[1] || S.L[2] != Dd.L[2])
        return set_err(QS3_ERR_INVALID_ARG, "source and target bases are on different lattices");
    if (Dd.nd != S.nd + 1) return set_err(QS3_ERR_INVALID_ARG, "target n_down must be source n_down + 1");
    if (S.has_k != Dd.has_k) return set_err(QS3_ERR_INVALID_ARG, "both bases need momenta, or neither");
    if (ss < 0 || ss >= S.S || sd < 0 || sd >= Dd.S) return set_err(QS3_ERR_INVALID_ARG, "sector index");
    if (S.has_k)
        for (int a = 0; a < 3; ++a)
            if ((((long long)S.K[3 * ss + a] + Q[a]) % S.L[a] + S.L[a]) % S.L[a] != Dd.K[3 * sd + a])
                return set_err(QS3_ERR_SYMMETRY, "target momentum is not K + Q (axis %d)", a);
    double2 *ph = nullptr;
    QS3_TRY(noalloc_scratch(st, &ph));
    if (Dd.dims[sd] == 0) return QS3_OK;
    if (S.dims[ss] == 0) {
        QS3_CUDA(cudaMemsetAsync(psi, 0, Dd.dims[sd] * 16, st));
        return QS3_OK;
    }
    // Q reduced into [0, L) first: the angle is unchanged and the integer
    // products of the phase kernel stay far below 2^63
    int Qr[3];
    for (int a = 0; a < 3; ++a) Qr[a] = (int)(((long long)Q[a] % S.L[a] + S.L[a]) % S.L[a]);
    k_site_phases<<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.L[0], S.L[1], S.L[2], Qr[0], Qr[1], Qr[2], ph);
    QS3_LAUNCHED();
    if (S.nd == 0) {
        k_smq_vac<<<(unsigned)((Dd.dims[sd] + 255) / 256), 256, 0, st>>>(Dd.secs[sd], Dd.has_k ? 1 : 0, S.N, ph,
                                                                          (const double2 *)phi, (double2 *)psi);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    return dispatch_smq(S, ss, Dd, sd, ph, (const double2 *)phi, (double2 *)psi, st);
}

}  // namespace qs3

extern "C" int qs3_smq_noalloc(qs3_basis_t src, int32_t s_src, const void *phi, qs3_basis_t dst, int32_t s_dst,
                               const int32_t *Q, void *psi, void *stream) {
    qs3::clear_err();
    if (!src || !dst || !phi || !psi || !Q) return qs3::set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    return qs3::smq_noalloc(src->B, s_src, phi, dst->B, s_dst, Q, psi, (cudaStream_t)stream);
}
