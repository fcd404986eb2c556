// qs3_hphi.cu -- the matrix-free product psi = H phi (Alg. 9 of the paper,
// with the readings: norm ratio sqrt(N_a'/N_a) of Eq. (hak2), pull-form phase
// e^{+ik.l} with T^l a' = a'_rep, hop amplitude Jxy/2 of Eq. (1)).
//
// GPU design: one thread per row (consecutive threads own consecutive ranks,
// so in the colex order the gathers phi[a'] of one hop class land close
// together), a persistent grid striding over 256-row tiles of all sectors of
// a basis, the binomial table and the site-coordinate table staged in shared
// memory, and no atomics.  Per row:
//   - unrank (Alg. 1) the row's rank, or the representative's rank sigma[row];
//   - diagonal: sum_b Jz_b/4 - (1/2) sum_{i in a} s_i + (down-down Jz) + field,
//     with s_i = sum_j Jz_ij folded into the per-site constant u_i;
//   - for each down spin i and each bond (i, j) with j empty: the hop target
//     is the sorted list with i replaced by j (Alg. 3); its rank (U(1)), or
//     its representative and stabiliser via the pruned translation search and
//     the two-level index over sigma (k-sectors, Alg. 7-9);
//   - accumulate in the vector's precision (fp32 or fp64), write psi once.
#include <algorithm>
#include <atomic>

#include "qs3_fixed.cuh"
#include "qs3_hphi_common.cuh"

namespace qs3 {


// TB (k-sectors): representative and row from the representative table
// (LatView::orb, SecView::t2) instead of the search and sigma lookup
template <int ND, typename VT, bool KS, bool TB = false>
__global__ void __launch_bounds__(NTHREADS, (KS && TB && sizeof(VT) == 16) ? 4 : 3) k_hphi(LatView L, const SecView *__restrict__ secs,
                                                   const int *__restrict__ tile0, int S, int ntiles,
                                                   const VT *__restrict__ phi, VT *__restrict__ psi,
                                                   const int *__restrict__ active) {
    using R = typename VTr<VT>::R;
    using CT = typename VTr<VT>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    SmemLayout sm = carve(L, smem);
    stage_tables(L, sm.sC, KS ? sm.sxyz : nullptr);
    R *snorm = (R *)sm.snorm;
    if (threadIdx.x < 9) {
        snorm[threadIdx.x] = (R)sqrt((double)threadIdx.x);
        snorm[9 + threadIdx.x] = threadIdx.x ? (R)(1.0 / sqrt((double)threadIdx.x)) : (R)0;
    }
    const R *jxy = jxy_table<VT>(L);
    __syncthreads();
    // persistent grid striding over the tiles of all sectors (better balanced
    // than contiguous per-block ranges, measured); a block restages the phase
    // table of its tile's sector when the sector changes
    CT *ph = (CT *)sm.sph;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s = (S == 1) ? 0 : sector_of_tile(tile0, S, t);
        if (active && !active[s]) continue;
        const SecView sv = secs[s];
        if (KS && s != cur) {
            __syncthreads();
            const CT *g = phase_table<CT>(sv);
            for (int i = threadIdx.x; i < L.N; i += blockDim.x) ph[i] = g[i];
            __syncthreads();
            cur = s;
        }
        const uint64_t row = (uint64_t)(t - sv.tile0) * TILE + threadIdx.x;
        if (row >= sv.dim) continue;
        const uint64_t rank = KS ? __ldg(sv.sigma + row) : row;
        int c[ND];
        unrank(rank, sm.sC, L.np1, c);
        const VT *ph_in = phi + sv.off;
        const VT x0 = ph_in[row];
        R rs = 0;
        int st_row = 1;
        if constexpr (KS) {
            st_row = sv.stab[row];
            rs = snorm[9 + st_row];
        }
        // diagonal in the vector precision: fp32 kernels keep off the fp64 unit
        R e = diag_c0<R>(L), dd = 0;
        CT acc;
        acc.x = 0; acc.y = 0;
        // k-sectors with one hop amplitude on every bond: sum phase x phi over
        // the hops and multiply by the amplitude once (two fp64 multiplies
        // fewer per hop)
        const R juni = (R)L.jh_uniform;
        const bool uni = KS && juni != (R)0;
        CT acch;
        acch.x = 0; acch.y = 0;
        // U(1), fp32, N_down <= 4: per occupied site, the ranks of its first
        // DEGB hop targets are formed first and their gathers then issue
        // together, so a thread keeps several independent loads in flight
        // (measured: 5% faster for fp32; the fp64 kernels run slower this way)
        constexpr bool BATCH = !KS && ND <= 4 && sizeof(R) == 4;
        constexpr int DEGB = 6;
        if constexpr (BATCH) {
#pragma unroll
            for (int m = 0; m < ND; ++m) {
                const int i = c[m];
                e += diag_u<R>(L, i);
                const int e0 = __ldg(L.adj_ptr + i), e1 = __ldg(L.adj_ptr + i + 1);
                uint64_t r2b[DEGB];
                R cfb[DEGB];
#pragma unroll
                for (int b = 0; b < DEGB; ++b) {
                    const int q = e0 + b;
                    cfb[b] = 0;
                    r2b[b] = 0;
                    if (q < e1) {
                        const int j = __ldg(L.adj_nbr + q);
                        bool occ = false;
#pragma unroll
                        for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                        if (occ) {
                            dd += diag_jz<R>(L, q);
                        } else {
                            const bool inplace = (m == 0 || j > c[m > 0 ? m - 1 : 0]) &&
                                                 (m == ND - 1 || j < c[m + 1 < ND ? m + 1 : m]);
                            if (inplace) {
                                r2b[b] = rank - sm.sC[(m + 1) * L.np1 + c[m]] + sm.sC[(m + 1) * L.np1 + j];
                            } else {
                                int tt[ND];
#pragma unroll
                                for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                                sort_net(tt);
                                r2b[b] = rank_of(tt, sm.sC, L.np1);
                            }
                            cfb[b] = __ldg(jxy + q);
                        }
                    }
                }
                VT vb[DEGB];
#pragma unroll
                for (int b = 0; b < DEGB; ++b)
                    if (cfb[b] != (R)0) vb[b] = ph_in[r2b[b]];
#pragma unroll
                for (int b = 0; b < DEGB; ++b)
                    if (cfb[b] != (R)0) madd_r(acc, cfb[b], vb[b]);
                // sites with more than DEGB neighbours: the rest one at a time
                for (int q = e0 + DEGB; q < e1; ++q) {
                    const int j = __ldg(L.adj_nbr + q);
                    bool occ = false;
#pragma unroll
                    for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                    if (occ) {
                        dd += diag_jz<R>(L, q);
                        continue;
                    }
                    int tt[ND];
#pragma unroll
                    for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                    sort_net(tt);
                    madd_r(acc, __ldg(jxy + q), ph_in[rank_of(tt, sm.sC, L.np1)]);
                }
            }
        }
        // the k-sector hop body (with the representative search) stays rolled:
        // unrolled N_down times it overflows the instruction cache (measured)
        constexpr int UNR = KS ? 1 : ND;
#pragma unroll UNR
        for (int m = 0; m < (BATCH ? 0 : ND); ++m) {
            const int i = pick(c, m);
            e += diag_u<R>(L, i);
            const int e0 = __ldg(L.adj_ptr + i), e1 = __ldg(L.adj_ptr + i + 1);
            // a hop to c_{m-1} < j < c_{m+1} keeps its place in the sorted list
            // (and lands on an empty site): its rank changes in the m-th term only
            const int lo = m > 0 ? pick(c, m > 0 ? m - 1 : 0) : -1;
            const int hi = m < ND - 1 ? pick(c, m < ND - 1 ? m + 1 : m) : L.np1;
            const uint64_t base = rank - sm.sC[(m + 1) * L.np1 + i];
            for (int q = e0; q < e1; ++q) {
                const int j = __ldg(L.adj_nbr + q);
                const bool inpl = j > lo && j < hi;
                if (!inpl) {
                    bool occ = false;
#pragma unroll
                    for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                    if (occ) {
                        dd += diag_jz<R>(L, q);
                        continue;
                    }
                }
                int tt[ND];
#pragma unroll
                for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                const R jh = __ldg(jxy + q);
                if constexpr (!KS) {
                    // j keeps position m when it stays between the neighbours of
                    // c_m: only the m-th term of the rank changes
                    const bool inplace = (m == 0 || j > c[m > 0 ? m - 1 : 0]) && (m == ND - 1 || j < c[m + 1 < ND ? m + 1 : m]);
                    uint64_t r2;
                    if (inplace) {
                        r2 = rank - sm.sC[(m + 1) * L.np1 + c[m]] + sm.sC[(m + 1) * L.np1 + j];
                    } else {
                        sort_net(tt);
                        r2 = rank_of(tt, sm.sC, L.np1);
                    }
                    madd_r(acc, jh, ph_in[r2]);
                } else {
                    uint32_t idx;
                    int u;
                    if constexpr (TB) {
                        uint64_t r2;
                        if (inpl) {
                            r2 = base + sm.sC[(m + 1) * L.np1 + j];
                        } else {
                            sort_net(tt);
                            r2 = rank_of(tt, sm.sC, L.np1);
                        }
                        const uint32_t e = __ldg(L.orb + r2);
                        if ((e >> 12) >= L.n_orb) continue;     // never for a complete table
                        const int32_t row2 = __ldg(sv.t2 + (e >> 12));
                        if (row2 < 0) continue;
                        idx = (uint32_t)row2;
                        u = (int)(e & 4095u);
                    } else {
                        int rep[ND];
                        int ax, by, cz;
                        const uint64_t r2 = canon(tt, L, sm.sxyz, sm.sC, rep, ax, by, cz);
                        if (!sigma_find(sv, prefix_of(rep, sm.sC, L.np1), r2, idx)) continue;
                        u = ax + L.L[0] * (by + L.L[1] * cz);
                    }
                    CT p = ph[u];   // generic load (L1-cached)
                    const int st = __ldg(sv.stab + idx);
                    if (uni) {
                        // uniform J^xy: the amplitude is applied once per row below
                        if (st != st_row) {
                            const R f = snorm[st] * rs;
                            p.x *= f;
                            p.y *= f;
                        }
                        acc_add(acch, p, ph_in[idx]);
                    } else {
                        const R w = (st == st_row) ? jh : jh * snorm[st] * rs;
                        p.x *= w;
                        p.y *= w;
                        acc_add(acc, p, ph_in[idx]);
                    }
                }
            }
        }
        if (KS && uni) madd_r(acc, juni, acch);
        madd_r(acc, e + (R)0.5 * dd, x0);
        store(psi + sv.off + row, acc);
    }
}

// H Phi of the binary64 engine on the integer units: k-sectors with the
// representative table and one hop amplitude J/2 on every bond.  phi comes
// twice: as binary64 (the diagonal term) and as its digit-store image (dg:
// the top-digit plane then the low-digit plane, D int2 (re, im) each; ge:
// the grid exponent of every chunk's warp groups).  Each hop's product
// phase x phi is formed exactly on the images (the phases on the grid 2^-52,
// staged per sector as digits) with mad.wide.s32, folded at weight 2^52
// (rounded to nearest) and added to the row sum (RowAcc); terms whose target
// stabiliser differs from the row's (norm ratio != 1, rare) are summed in
// binary64 as in k_hphi.  The row sum is rounded to binary64 once, then
// psi = J/2 sum + diag phi in binary64.  Graph mode (dx): dg and ge are the
// store's, slot *dx.
// the row sum of the integer H Phi: (re, im) 2^(r - 1075), r the group
// exponent of the largest term so far; a term T 2^(em - 1075) (|T| <= 2^54)
// is rounded to nearest onto that grid, and a term of a coarser group first
// moves the sum to its grid.  With at most 48 terms |sum| < 2^60, and the
// error is at most (terms + moves) / 2 units of the final grid, i.e. about
// 2^-54 of the largest term each (binary64 accumulation: 2^-53 of each
// partial sum).
struct RowAcc {
    long long re = 0, im = 0;
    int r = -100000;
};
__device__ __forceinline__ long long rshift_round(long long x, int d) {
    if (d <= 0) return x;
    if (d > 62) return 0;
    return (x + (1ll << (d - 1))) >> d;
}
__device__ __forceinline__ void row_add(RowAcc &a, long long tr, long long ti, int em) {
    if (em > a.r) {
        const int d = min(em - a.r, 63);
        a.re = rshift_round(a.re, d);
        a.im = rshift_round(a.im, d);
        a.r = em;
    }
    const int d = a.r - em;
    a.re += rshift_round(tr, d);
    a.im += rshift_round(ti, d);
}
// the term phase x phi on the digits: (pr + i pi)(fr + i fi), folded at
// weight 2^52 (rounded to nearest): units 2^(em - 1075) for phi on the grid
// of em and the phase on 2^-52
__device__ __forceinline__ void term_x(int4 p, int2 f1, int2 f0, long long &tr, long long &ti) {
    const long long hr = mad_w(p.x, f1.x, 0), hn = mad_w(p.z, f1.y, 0);
    const long long mr = mad_w(p.x, f0.x, mad_w(p.y, f1.x, 0));
    const long long mn = mad_w(p.z, f0.y, mad_w(p.w, f1.y, 0));
    const long long hi = mad_w(p.x, f1.y, mad_w(p.z, f1.x, 0));
    const long long mi = mad_w(p.x, f0.y, mad_w(p.y, f1.y, mad_w(p.z, f0.x, mad_w(p.w, f1.x, 0))));
    tr = (hr - hn) + ((mr - mn + (1ll << 25)) >> 26);
    ti = hi + ((mi + (1ll << 25)) >> 26);
}

template <int ND>
__global__ void __launch_bounds__(NTHREADS, 4) k_hphi_x(LatView L, const SecView *__restrict__ secs,
                                                       const int *__restrict__ tile0, int S, int ntiles,
                                                       const double2 *__restrict__ phi, const int2 *__restrict__ dg,
                                                       const int *__restrict__ ge, const int *__restrict__ chunk0,
                                                       int nchunks, uint64_t D,
                                                       const int *__restrict__ dx, double2 *__restrict__ psi,
                                                       const int *__restrict__ active) {
    extern __shared__ __align__(16) unsigned char smem[];
    SmemLayout sm = carve(L, smem);
    stage_tables(L, sm.sC, sm.sxyz);
    double *snorm = (double *)sm.snorm;
    if (threadIdx.x < 9) {
        snorm[threadIdx.x] = sqrt((double)threadIdx.x);
        snorm[9 + threadIdx.x] = threadIdx.x ? 1.0 / sqrt((double)threadIdx.x) : 0.0;
    }
    if (dx) {
        dg += (uint64_t)(*dx) * 2 * D;
        ge += (uint64_t)(*dx) * nchunks * XW;
    }
    const double juni = L.jh_uniform;
    __syncthreads();
    int4 *pd = (int4 *)sm.sph;          // the current sector's phases: (re.P1, re.P0, im.P1, im.P0) on 2^-52
    int cur = -1, c0s = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s = (S == 1) ? 0 : sector_of_tile(tile0, S, t);
        if (active && !active[s]) continue;
        const SecView sv = secs[s];
        if (s != cur) {
            __syncthreads();
            for (int i = threadIdx.x; i < L.N; i += blockDim.x) {
                const double2 p = sv.ph64[i];
                int a1, a0, b1, b0;
                fx_digits((uint32_t)__double2hiint(p.x), (uint32_t)__double2loint(p.x), 1023, a1, a0);
                fx_digits((uint32_t)__double2hiint(p.y), (uint32_t)__double2loint(p.y), 1023, b1, b0);
                pd[i] = make_int4(a1, a0, b1, b0);
            }
            c0s = chunk0[s];
            __syncthreads();
            cur = s;
        }
        const uint64_t row = (uint64_t)(t - sv.tile0) * TILE + threadIdx.x;
        if (row >= sv.dim) continue;
        const uint64_t rank = __ldg(sv.sigma + row);
        int c[ND];
        unrank(rank, sm.sC, L.np1, c);
        const double2 x0 = phi[sv.off + row];
        const int st_row = sv.stab[row];
        const double rs = snorm[9 + st_row];
        double e = L.c0, dd = 0.0;
        RowAcc acc;
        double2 acc64 = make_double2(0.0, 0.0);
#pragma unroll 1
        for (int m = 0; m < ND; ++m) {
            const int i = pick(c, m);
            e += diag_u<double>(L, i);
            const int e0 = __ldg(L.adj_ptr + i), e1 = __ldg(L.adj_ptr + i + 1);
            // a hop to c_{m-1} < j < c_{m+1} keeps its place in the sorted list
            const int lo = m > 0 ? pick(c, m > 0 ? m - 1 : 0) : -1;
            const int hi = m < ND - 1 ? pick(c, m < ND - 1 ? m + 1 : m) : L.np1;
            const uint64_t base = rank - sm.sC[(m + 1) * L.np1 + i];
            for (int q = e0; q < e1; ++q) {
                const int j = __ldg(L.adj_nbr + q);
                const bool inpl = j > lo && j < hi;
                if (!inpl) {
                    bool occ = false;
#pragma unroll
                    for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                    if (occ) {
                        dd += diag_jz<double>(L, q);
                        continue;
                    }
                }
                uint64_t r2;
                if (inpl) {
                    r2 = base + sm.sC[(m + 1) * L.np1 + j];
                } else {
                    int tt[ND];
#pragma unroll
                    for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                    sort_net(tt);
                    r2 = rank_of(tt, sm.sC, L.np1);
                }
                const uint32_t ee = __ldg(L.orb + r2);
                if ((ee >> 12) >= L.n_orb) continue;     // never for a complete table
                const int32_t row2 = __ldg(sv.t2 + (ee >> 12));
                if (row2 < 0) continue;
                const uint32_t idx = (uint32_t)row2;
                const int u = (int)(ee & 4095u);
                const int st = __ldg(sv.stab + idx);
                if (st == st_row) {
                    const uint64_t gi = sv.off + idx;
                    const int2 f1 = dg[gi], f0 = dg[D + gi];
                    const int em = __ldg(ge + (uint64_t)(c0s + (int)(idx >> 11)) * XW + dg_group((int)(idx & 2047u)));
                    long long tr, ti;
                    term_x(pd[u], f1, f0, tr, ti);
                    row_add(acc, tr, ti, em);
                } else {
                    double2 p = sv.ph64[u];
                    const double f = snorm[st] * rs;
                    p.x *= f;
                    p.y *= f;
                    acc_add(acc64, p, phi[sv.off + idx]);
                }
            }
        }
        double2 acch;
        acch.x = i128_ldexp(acc.re, acc.r - 1075) + acc64.x;
        acch.y = i128_ldexp(acc.im, acc.r - 1075) + acc64.y;
        const double ed = e + 0.5 * dd;
        double2 out;
        out.x = fma(ed, x0.x, juni * acch.x);
        out.y = fma(ed, x0.y, juni * acch.y);
        psi[sv.off + row] = out;
    }
}

// The same product batched over sectors (all momenta of one basis share the
// orbits and their hops; only the phases and the rows differ): one thread per
// (orbit g, group of OSG sectors) unranks g's representative once, lists its
// hop targets (orbit, translation, |Stab|) and its diagonal once, then forms
// g's row in each sector of the group from them: per term one row lookup,
// the digits of the target and its group exponent, the exact product with
// the sector's phase digits and the row sum, as in k_hphi_x (whose output it
// reproduces bit for bit: the terms come in the same order).  The hop lists
// live in shared memory, maxh entries per thread.
constexpr int OSG = 8;

template <int ND>
__global__ void __launch_bounds__(NTHREADS) k_hphi_o(LatView L, const SecView *__restrict__ secs, int S,
                                                   const uint64_t *__restrict__ oreps,
                                                   const uint8_t *__restrict__ ostab, uint32_t n_orb, int ngrp,
                                                   const int4 *__restrict__ phdig, const double2 *__restrict__ phi,
                                                   const int2 *__restrict__ dg, const int *__restrict__ ge,
                                                   const int *__restrict__ chunk0, int nchunks, uint64_t D,
                                                   const int *__restrict__ dx,
                                                   double2 *__restrict__ psi, const int *__restrict__ active,
                                                   int maxh) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sC = (uint64_t *)smem;
    double *snorm = (double *)(sC + (L.nd + 3) * L.np1);
    uint32_t *hl = (uint32_t *)(snorm + 18);                     // hop targets g2 << 12 | u
    uint8_t *hs = (uint8_t *)(hl + (size_t)maxh * blockDim.x);     // their |Stab|
    for (int i = threadIdx.x; i < (L.nd + 3) * L.np1; i += blockDim.x) sC[i] = L.binom[i];
    if (threadIdx.x < 9) {
        snorm[threadIdx.x] = sqrt((double)threadIdx.x);
        snorm[9 + threadIdx.x] = threadIdx.x ? 1.0 / sqrt((double)threadIdx.x) : 0.0;
    }
    if (dx) {
        dg += (uint64_t)(*dx) * 2 * D;
        ge += (uint64_t)(*dx) * nchunks * XW;
    }
    __syncthreads();
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (uint64_t)n_orb * ngrp) return;
    const uint32_t g = (uint32_t)(tid % n_orb);
    const int grp = (int)(tid / n_orb);
    const int s_lo = grp * OSG, s_hi = min(S, s_lo + OSG);
    bool any = false;
    for (int s = s_lo; s < s_hi; ++s) any |= (!active || active[s]) && __ldg(secs[s].t2 + g) >= 0;
    if (!any) return;
    uint32_t *my = hl + threadIdx.x;                             // entry h at my[h * blockDim.x]
    uint8_t *mys = hs + threadIdx.x;
    const uint64_t rank = __ldg(oreps + g);
    int c[ND];
    unrank(rank, sC, L.np1, c);
    const int st_row = __ldg(ostab + g);
    const double rs = snorm[9 + st_row];
    double e = L.c0, dd = 0.0;
    int nh = 0;
#pragma unroll 1
    for (int m = 0; m < ND; ++m) {
        const int i = pick(c, m);
        e += diag_u<double>(L, i);
        const int e0 = __ldg(L.adj_ptr + i), e1 = __ldg(L.adj_ptr + i + 1);
        const int lo = m > 0 ? pick(c, m > 0 ? m - 1 : 0) : -1;
        const int hi = m < ND - 1 ? pick(c, m < ND - 1 ? m + 1 : m) : L.np1;
        const uint64_t base = rank - sC[(m + 1) * L.np1 + i];
        for (int q = e0; q < e1; ++q) {
            const int j = __ldg(L.adj_nbr + q);
            const bool inpl = j > lo && j < hi;
            if (!inpl) {
                bool occ = false;
#pragma unroll
                for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                if (occ) {
                    dd += diag_jz<double>(L, q);
                    continue;
                }
            }
            uint64_t r2;
            if (inpl) {
                r2 = base + sC[(m + 1) * L.np1 + j];
            } else {
                int tt[ND];
#pragma unroll
                for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                sort_net(tt);
                r2 = rank_of(tt, sC, L.np1);
            }
            const uint32_t ee = __ldg(L.orb + r2);
            if ((ee >> 12) >= n_orb) continue;                   // never for a complete table
            my[(size_t)nh * blockDim.x] = ee;
            mys[(size_t)nh * blockDim.x] = __ldg(ostab + (ee >> 12));
            ++nh;
        }
    }
    const double ed = e + 0.5 * dd;
    const double juni = L.jh_uniform;
    for (int s = s_lo; s < s_hi; ++s) {
        if (active && !active[s]) continue;
        const int32_t *t2 = secs[s].t2;
        const int32_t row = __ldg(t2 + g);
        if (row < 0) continue;
        const uint64_t off = secs[s].off;
        const int c0s = __ldg(chunk0 + s);
        const int4 *pds = phdig + (size_t)s * L.N;
        RowAcc acc;
        double2 acc64 = make_double2(0.0, 0.0);
        // four terms at a time: their row lookups, then their digit gathers,
        // are in flight together; the terms are added in list order
        for (int h0 = 0; h0 < nh; h0 += 4) {
            uint32_t ee[4];
            int32_t r2[4];
            int stb[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const bool in = h0 + b < nh;
                ee[b] = in ? my[(size_t)(h0 + b) * blockDim.x] : 0u;
                stb[b] = in ? mys[(size_t)(h0 + b) * blockDim.x] : 0;
                r2[b] = in ? __ldg(t2 + (ee[b] >> 12)) : -1;
            }
            int2 f1[4], f0[4];
            int em[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (r2[b] >= 0 && stb[b] == st_row) {
                    const uint64_t gi = off + (uint32_t)r2[b];
                    f1[b] = dg[gi];
                    f0[b] = dg[D + gi];
                    em[b] = __ldg(ge + (uint64_t)(c0s + (r2[b] >> 11)) * XW + dg_group(r2[b] & 2047));
                } else {
                    f1[b] = f0[b] = make_int2(0, 0);
                    em[b] = 0;
                }
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (r2[b] < 0) continue;
                const int u = (int)(ee[b] & 4095u);
                if (stb[b] == st_row) {
                    long long tr, ti;
                    term_x(__ldg(pds + u), f1[b], f0[b], tr, ti);
                    row_add(acc, tr, ti, em[b]);
                } else {
                    double2 p = secs[s].ph64[u];
                    const double f = snorm[stb[b]] * rs;
                    p.x *= f;
                    p.y *= f;
                    acc_add(acc64, p, phi[off + (uint32_t)r2[b]]);
                }
            }
        }
        double2 acch;
        acch.x = i128_ldexp(acc.re, acc.r - 1075) + acc64.x;
        acch.y = i128_ldexp(acc.im, acc.r - 1075) + acc64.y;
        const double2 x0 = phi[off + (uint32_t)row];
        double2 out;
        out.x = fma(ed, x0.x, juni * acch.x);
        out.y = fma(ed, x0.y, juni * acch.y);
        psi[off + (uint32_t)row] = out;
    }
}

// U(1) H Phi with 32-bit ranks, for C(N, N_down) < 2^32, N_down <= 4, fp32
// vectors and lattices of degree <= 6: the binomial rows 0..N_down as a
// 32-bit table in shared memory, one thread per row striding over the single
// sector, and the fixed-width adjacency (DEGB = 4 or 6 entries per site, a
// site with fewer padded with itself and zero couplings), one 8-byte load
// per entry (neighbour, hop amplitude).  The hop of c_m to j keeps its place
// in the sorted list when c_{m-1} < j < c_{m+1}; then its rank is the row's
// rank with C(c_m, m+1) replaced by C(j, m+1) -- two compares and one table
// read, and a padded entry (j = c_m) lands on the row itself with amplitude
// 0.  Only the other hops (j occupied, or j passing another down spin) take
// the occupancy test and the re-sort.  Per occupied site the ranks of its
// DEGB entries are formed before their gathers issue together.  Same
// signature as k_hphi (the launch and the autotuner treat both alike).
template <int ND, typename VT, int DEGB>
__global__ void __launch_bounds__(NTHREADS, DEGB <= 4 ? 6 : 4) k_hphi_u1n(LatView L, const SecView *__restrict__ secs,
                                                      const int *__restrict__ tile0, int S, int ntiles,
                                                      const VT *__restrict__ phi, VT *__restrict__ psi,
                                                      const int *__restrict__ active) {
    using R = typename VTr<VT>::R;
    using CT = typename VTr<VT>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *sC = (uint32_t *)smem;
    const int np1 = L.np1;
    for (int i = threadIdx.x; i < (ND + 1) * np1; i += blockDim.x) sC[i] = (uint32_t)L.binom[i];
    __syncthreads();
    if (active && !active[0]) return;
    const uint64_t dim = secs[0].dim;     // < 2^32
    const int2 *__restrict__ pad = L.adj_pad;
    for (uint64_t rw = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; rw < dim; rw += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t row = (uint32_t)rw;
        int c[ND];
        unrank32(row, sC, np1, c);
        const VT x0 = phi[row];
        R e = diag_c0<R>(L), dd = 0;
        CT acc;
        acc.x = 0; acc.y = 0;
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            const int i = c[m];
            e += diag_u<R>(L, i);
            const int lo = m > 0 ? c[m > 0 ? m - 1 : 0] : -1;
            const int hi = m < ND - 1 ? c[m < ND - 1 ? m + 1 : m] : np1;
            const uint32_t base = row - sC[(m + 1) * np1 + i];
            const uint32_t *col = sC + (m + 1) * np1;
            uint32_t r2b[DEGB];
            R cfb[DEGB];
#pragma unroll
            for (int b = 0; b < DEGB; ++b) {
                const int2 pk = __ldg(pad + i * DEGB + b);
                const int j = pk.x;
                const R cf = (R)__int_as_float(pk.y);
                r2b[b] = base + col[j];
                cfb[b] = cf;
                if (!(j > lo && j < hi)) {
                    // occupied, or passing another down spin
                    bool occ = false;
#pragma unroll
                    for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                    if (occ) {
                        dd += (R)__ldg(L.adj_jz_pad + i * DEGB + b);
                        cfb[b] = 0;
                        r2b[b] = row;
                    } else {
                        int tt[ND];
#pragma unroll
                        for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                        sort_net(tt);
                        r2b[b] = rank_of32(tt, sC, np1);
                    }
                }
            }
            VT vb[DEGB];
#pragma unroll
            for (int b = 0; b < DEGB; ++b) vb[b] = phi[r2b[b]];
#pragma unroll
            for (int b = 0; b < DEGB; ++b) madd_r(acc, cfb[b], vb[b]);
        }
        madd_r(acc, e + (R)0.5 * dd, x0);
        store(psi + row, acc);
    }
}

// nnz count per sector: the diagonal plus every hop that lands on a member of the sector
template <int ND, bool KS>
__global__ void __launch_bounds__(NTHREADS) k_count(LatView L, const SecView *__restrict__ secs,
                                                    const int *__restrict__ tile0, int S, int ntiles,
                                                    unsigned long long *out) {
    extern __shared__ __align__(16) unsigned char smem[];
    SmemLayout sm = carve(L, smem);
    stage_tables(L, sm.sC, KS ? sm.sxyz : nullptr);
    __syncthreads();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s = (S == 1) ? 0 : sector_of_tile(tile0, S, t);
        const SecView sv = secs[s];
        const uint64_t row = (uint64_t)(t - sv.tile0) * TILE + threadIdx.x;
        unsigned long long cnt = 0;
        if (row < sv.dim) {
            const uint64_t rank = KS ? sv.sigma[row] : row;
            int c[ND];
            unrank(rank, sm.sC, L.np1, c);
            cnt = 1;
#pragma unroll
            for (int m = 0; m < ND; ++m) {
                const int i = c[m];
                for (int q = L.adj_ptr[i]; q < L.adj_ptr[i + 1]; ++q) {
                    const int j = L.adj_nbr[q];
                    bool occ = false;
#pragma unroll
                    for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                    if (occ) continue;
                    if constexpr (!KS) {
                        ++cnt;
                    } else {
                        int tt[ND];
#pragma unroll
                        for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                        int rep[ND];
                        int ax, by, cz;
                        const uint64_t r2 = canon(tt, L, sm.sxyz, sm.sC, rep, ax, by, cz);
                        uint32_t idx;
                        if (sigma_find(sv, prefix_of(rep, sm.sC, L.np1), r2, idx)) ++cnt;
                    }
                }
            }
        }
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out + s, cnt);
    }
}

// N_down = 0: H is the constant c0 on the single vacuum state of each sector
template <typename VT>
__global__ void k_diag0(double c0, uint64_t n, const VT *__restrict__ phi, VT *__restrict__ psi) {
    using R = typename VTr<VT>::R;
    using CT = typename VTr<VT>::C;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        CT acc; acc.x = 0; acc.y = 0;
        madd_r(acc, (R)c0, phi[i]);
        store(psi + i, acc);
    }
}


template <typename VT> struct DtIdx;
template <> struct DtIdx<float> { static constexpr int v = QS3_F32; };
template <> struct DtIdx<double> { static constexpr int v = QS3_F64; };
template <> struct DtIdx<float2> { static constexpr int v = QS3_C64; };
template <> struct DtIdx<double2> { static constexpr int v = QS3_C128; };

template <typename VT, typename KF>
static int tune_grid(KF kern, Basis &B, int occ, cudaStream_t st, const VT *phi, VT *psi, const int *active,
                     int &best_bps, size_t smem = (size_t)-1) {
    if (smem == (size_t)-1) smem = B.smem_bytes;
    return tune_blocks(B, occ, st, best_bps, [&](int grid) {
        kern<<<grid, NTHREADS, smem, st>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(), B.S, B.ntiles, phi, psi,
                                           active);
    });
}

template <int ND, typename VT, bool KS, bool TB>
static int hphi_ndt(Basis &B, const void *phi, void *psi, cudaStream_t st, const int *active) {
    static std::atomic<unsigned long long> cache{0};
    int grid = 1, occ = 1;
    QS3_TRY(launch_rows(k_hphi<ND, VT, KS, TB>, B, B.smem_bytes, cache, &grid, &occ));
    if (B.ntiles == 0) return QS3_OK;
    int &bps = B.tune_hphi[DtIdx<VT>::v];
    if (bps == 0) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        QS3_CUDA(cudaStreamIsCapturing(st, &cst));
        if (cst == cudaStreamCaptureStatusNone) {
            int b = occ;
            QS3_TRY(tune_grid(k_hphi<ND, VT, KS, TB>, B, occ, st, (const VT *)phi, (VT *)psi, active, b));
            bps = b;
        }
    }
    if (bps > 0) grid = std::max(1, std::min(B.ntiles, std::min(bps, occ) * num_sms()));
    k_hphi<ND, VT, KS, TB><<<grid, NTHREADS, B.smem_bytes, st>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(),
                                                                  B.S, B.ntiles, (const VT *)phi, (VT *)psi, active);
    QS3_LAUNCHED();
    return QS3_OK;
}

template <int ND, typename VT, int DEGB>
static int hphi_u1n(Basis &B, const void *phi, void *psi, cudaStream_t st, const int *active) {
    static std::atomic<unsigned long long> cache{0};
    const size_t smem = (size_t)(ND + 1) * (B.N + 1) * sizeof(uint32_t);
    int grid = 1, occ = 1;
    QS3_TRY(launch_rows(k_hphi_u1n<ND, VT, DEGB>, B, smem, cache, &grid, &occ));
    if (B.ntiles == 0) return QS3_OK;
    int &bps = B.tune_hphi[DtIdx<VT>::v];
    if (bps == 0) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        QS3_CUDA(cudaStreamIsCapturing(st, &cst));
        if (cst == cudaStreamCaptureStatusNone) {
            int b = occ;
            QS3_TRY(tune_grid(k_hphi_u1n<ND, VT, DEGB>, B, occ, st, (const VT *)phi, (VT *)psi, active, b, smem));
            bps = b;
        }
    }
    if (bps > 0) grid = std::max(1, std::min(B.ntiles, std::min(bps, occ) * num_sms()));
    k_hphi_u1n<ND, VT, DEGB><<<grid, NTHREADS, smem, st>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(), B.S,
                                                           B.ntiles, (const VT *)phi, (VT *)psi, active);
    QS3_LAUNCHED();
    return QS3_OK;
}

template <int ND, typename VT, bool KS>
static int hphi_nd(Basis &B, const void *phi, void *psi, cudaStream_t st, const int *active) {
    if constexpr (KS) {
        if (B.lv.orb) return hphi_ndt<ND, VT, true, true>(B, phi, psi, st, active);
    } else if constexpr (ND <= 4 && sizeof(typename VTr<VT>::R) == 4) {
        if (B.narrow_ranks && B.lv.pad_w == 4) return hphi_u1n<ND, VT, 4>(B, phi, psi, st, active);
        if (B.narrow_ranks && B.lv.pad_w == 6) return hphi_u1n<ND, VT, 6>(B, phi, psi, st, active);
    }
    return hphi_ndt<ND, VT, KS, false>(B, phi, psi, st, active);
}

template <typename VT, bool KS>
static int hphi_vt(Basis &B, const void *phi, void *psi, cudaStream_t st, const int *a) {
    switch (B.nd) {
        case 1: return hphi_nd<1, VT, KS>(B, phi, psi, st, a);
        case 2: return hphi_nd<2, VT, KS>(B, phi, psi, st, a);
        case 3: return hphi_nd<3, VT, KS>(B, phi, psi, st, a);
        case 4: return hphi_nd<4, VT, KS>(B, phi, psi, st, a);
        case 5: return hphi_nd<5, VT, KS>(B, phi, psi, st, a);
        case 6: return hphi_nd<6, VT, KS>(B, phi, psi, st, a);
        case 7: return hphi_nd<7, VT, KS>(B, phi, psi, st, a);
        case 8: return hphi_nd<8, VT, KS>(B, phi, psi, st, a);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

template <int ND>
static int hphix_nd(Basis &B, const double2 *phi, const int2 *dg, const int *ge, const int *dx,
                    double2 *psi, cudaStream_t st, const int *active) {
    static std::atomic<unsigned long long> cache{0};
    int grid = 1, occ = 1;
    QS3_TRY(launch_rows(k_hphi_x<ND>, B, B.smem_bytes, cache, &grid, &occ));
    if (B.ntiles == 0) return QS3_OK;
    auto launch = [&](int g) {
        k_hphi_x<ND><<<g, NTHREADS, B.smem_bytes, st>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(), B.S,
                                                         B.ntiles, phi, dg, ge, B.d_chunk0.as<int>(), B.nchunks,
                                                         B.total, dx, psi, active);
    };
    int &bps = B.tune_hphix;
    if (bps == 0) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        QS3_CUDA(cudaStreamIsCapturing(st, &cst));
        if (cst == cudaStreamCaptureStatusNone && !dx) {
            int b = occ;
            QS3_TRY(tune_blocks(B, occ, st, b, launch));
            bps = b;
        }
    }
    if (bps > 0) grid = std::max(1, std::min(B.ntiles, std::min(bps, occ) * num_sms()));
    launch(grid);
    QS3_LAUNCHED();
    return QS3_OK;
}

template <int ND>
static int hphio_nd(Basis &B, const double2 *phi, const int2 *dg, const int *ge, const int *dx,
                    double2 *psi, cudaStream_t st, const int *active) {
    const int maxh = std::max(1, B.nd * B.max_degree);
    const size_t smem = (size_t)(B.nd + 3) * (B.N + 1) * 8 + 18 * 8 + (size_t)maxh * NTHREADS * 5;
    if (smem > (size_t)MAX_DYN_SMEM) return set_err(QS3_ERR_OVERFLOW, "hop lists of %d entries per row", maxh);
    static std::atomic<int> attr{0};
    if (attr.load(std::memory_order_acquire) == 0) {
        QS3_CUDA(cudaFuncSetAttribute(k_hphi_o<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        attr.store(1, std::memory_order_release);
    }
    const int ngrp = (B.S + OSG - 1) / OSG;
    const uint64_t nthr = B.n_orb * (uint64_t)ngrp;
    if (nthr == 0) return QS3_OK;
    const int grid = (int)((nthr + NTHREADS - 1) / NTHREADS);
    k_hphi_o<ND><<<grid, NTHREADS, smem, st>>>(B.lv, B.d_secs.as<SecView>(), B.S, B.d_oreps.as<uint64_t>(),
                                                B.d_ostab.as<uint8_t>(), (uint32_t)B.n_orb, ngrp,
                                                B.d_phdig.as<int4>(), phi, dg, ge, B.d_chunk0.as<int>(), B.nchunks,
                                                B.total, dx, psi, active, maxh);
    QS3_LAUNCHED();
    return QS3_OK;
}

bool hphi_x_ok(const Basis &B) {
    return B.has_k && B.lv.orb && B.lv.jh_uniform != 0.0 && B.nd > 0 && !B.stored_terms && B.total > 0;
}

int hphi_x_launch(Basis &B, const void *phi, const void *dg, const int *ge, const int *dx, void *psi, cudaStream_t st,
                  const int *active) {
    if (!hphi_x_ok(B)) return set_err(QS3_ERR_STATE, "the integer H Phi needs a k-sector basis with the "
                                                     "representative table and one hop amplitude");
    const double2 *p = (const double2 *)phi;
    const int2 *g = (const int2 *)dg;
    double2 *o = (double2 *)psi;
    // several sectors share the orbits: the orbit-batched kernel
    if (B.S >= 2 && B.d_oreps.p) {
        switch (B.nd) {
            case 1: return hphio_nd<1>(B, p, g, ge, dx, o, st, active);
            case 2: return hphio_nd<2>(B, p, g, ge, dx, o, st, active);
            case 3: return hphio_nd<3>(B, p, g, ge, dx, o, st, active);
            case 4: return hphio_nd<4>(B, p, g, ge, dx, o, st, active);
            case 5: return hphio_nd<5>(B, p, g, ge, dx, o, st, active);
            case 6: return hphio_nd<6>(B, p, g, ge, dx, o, st, active);
            case 7: return hphio_nd<7>(B, p, g, ge, dx, o, st, active);
            case 8: return hphio_nd<8>(B, p, g, ge, dx, o, st, active);
            default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
        }
    }
    switch (B.nd) {
        case 1: return hphix_nd<1>(B, p, g, ge, dx, o, st, active);
        case 2: return hphix_nd<2>(B, p, g, ge, dx, o, st, active);
        case 3: return hphix_nd<3>(B, p, g, ge, dx, o, st, active);
        case 4: return hphix_nd<4>(B, p, g, ge, dx, o, st, active);
        case 5: return hphix_nd<5>(B, p, g, ge, dx, o, st, active);
        case 6: return hphix_nd<6>(B, p, g, ge, dx, o, st, active);
        case 7: return hphix_nd<7>(B, p, g, ge, dx, o, st, active);
        case 8: return hphix_nd<8>(B, p, g, ge, dx, o, st, active);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

int hphi_launch(Basis &B, qs3_dtype dt, const void *phi, void *psi, cudaStream_t st, const int *active) {
    if (!phi || !psi) return set_err(QS3_ERR_INVALID_ARG, "NULL vector");
    if (phi == psi) return set_err(QS3_ERR_INVALID_ARG, "phi and psi alias");
    if (dt == QS3_C128DF) return hphi_df_launch(B, phi, nullptr, 0, psi, st, active);
    if (dt == QS3_C128X) return hphi_x_binary64(B, phi, psi, st);
    if (B.has_k && (dt == QS3_F32 || dt == QS3_F64))
        return set_err(QS3_ERR_STATE, "k-sector bases need complex vectors (C64/C128)");
    if (B.total == 0) return QS3_OK;
    if (B.nd == 0) {
        const int grid = (int)std::min<uint64_t>((B.total + 255) / 256, 1024);
        switch (dt) {
            case QS3_F32: k_diag0<float><<<grid, 256, 0, st>>>(B.lv.c0, B.total, (const float *)phi, (float *)psi); break;
            case QS3_F64: k_diag0<double><<<grid, 256, 0, st>>>(B.lv.c0, B.total, (const double *)phi, (double *)psi); break;
            case QS3_C64: k_diag0<float2><<<grid, 256, 0, st>>>(B.lv.c0, B.total, (const float2 *)phi, (float2 *)psi); break;
            case QS3_C128: k_diag0<double2><<<grid, 256, 0, st>>>(B.lv.c0, B.total, (const double2 *)phi, (double2 *)psi); break;
            default: return set_err(QS3_ERR_INVALID_ARG, "dtype %d", (int)dt);
        }
        QS3_LAUNCHED();
        return QS3_OK;
    }
    if (B.has_k) {
        if (B.stored_terms && (dt == QS3_C64 || dt == QS3_C128)) return hphi_stored_launch(B, dt, phi, psi, st, active);
        if (dt == QS3_C64) return hphi_vt<float2, true>(B, phi, psi, st, active);
        if (dt == QS3_C128) return hphi_vt<double2, true>(B, phi, psi, st, active);
    } else {
        if (dt == QS3_F32) return hphi_vt<float, false>(B, phi, psi, st, active);
        if (dt == QS3_F64) return hphi_vt<double, false>(B, phi, psi, st, active);
        if (dt == QS3_C64) return hphi_vt<float2, false>(B, phi, psi, st, active);
        if (dt == QS3_C128) return hphi_vt<double2, false>(B, phi, psi, st, active);
    }
    return set_err(QS3_ERR_INVALID_ARG, "dtype %d", (int)dt);
}

template <int ND, bool KS>
static int count_nd(Basis &B, unsigned long long *d_out) {
    static std::atomic<unsigned long long> cache{0};
    int grid = 1;
    QS3_TRY(launch_rows(k_count<ND, KS>, B, B.smem_bytes, cache, &grid));
    k_count<ND, KS><<<grid, NTHREADS, B.smem_bytes>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(), B.S,
                                                       B.ntiles, d_out);
    QS3_LAUNCHED();
    return QS3_OK;
}

template <bool KS>
static int count_ks(Basis &B, unsigned long long *d_out) {
    switch (B.nd) {
        case 1: return count_nd<1, KS>(B, d_out);
        case 2: return count_nd<2, KS>(B, d_out);
        case 3: return count_nd<3, KS>(B, d_out);
        case 4: return count_nd<4, KS>(B, d_out);
        case 5: return count_nd<5, KS>(B, d_out);
        case 6: return count_nd<6, KS>(B, d_out);
        case 7: return count_nd<7, KS>(B, d_out);
        case 8: return count_nd<8, KS>(B, d_out);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

int count_nnz(Basis &B, uint64_t *nnz) {
    if (!B.nnz_valid) {
        B.nnz_sec.assign(B.S, 0);
        if (B.nd == 0 || B.total == 0) {
            for (int s = 0; s < B.S; ++s) B.nnz_sec[s] = B.dims[s];
        } else {
            DevBuf d;
            QS3_TRY(d.alloc(8 * (size_t)B.S));
            QS3_CUDA(cudaMemset(d.p, 0, 8 * (size_t)B.S));
            QS3_TRY(B.has_k ? count_ks<true>(B, d.as<unsigned long long>())
                            : count_ks<false>(B, d.as<unsigned long long>()));
            QS3_CUDA(cudaMemcpy(B.nnz_sec.data(), d.p, 8 * (size_t)B.S, cudaMemcpyDeviceToHost));
        }
        B.nnz = 0;
        for (uint64_t v : B.nnz_sec) B.nnz += v;
        B.nnz_valid = true;
    }
    *nnz = B.nnz;
    return QS3_OK;
}

}  // namespace qs3

extern "C" int qs3_hphi(qs3_basis_t b, qs3_dtype dtype, const void *phi, void *psi, void *stream) {
    qs3::clear_err();
    if (!b) return qs3::set_err(QS3_ERR_INVALID_ARG, "basis is NULL");
    return qs3::hphi_launch(b->B, dtype, phi, psi, (cudaStream_t)stream);
}
