// qs3_hphi_df.cu -- psi = H phi for k-sector vectors held in double-float
// form (QS3_C128DF): element r of phi is four floats (re.hi, re.lo, im.hi,
// im.lo) with re = re.hi + re.lo, im = im.hi + im.lo.  The terms are those of
// the complex128 product in qs3_hphi.cu (Alg. 9 with the same readings: norm
// ratio sqrt(|Stab a'| / |Stab a|), pull-form phase e^{+ik.l}, hop amplitude
// J^xy/2 of Eq. (1)), but every product and sum runs on the fp32 units as an
// error-free product (fma) and two-sum.  psi is written in complex128.
//
// Why: GB300 retires about one fp64 fused multiply-add per SM and clock
// against 128 in fp32, so the complex128 kernel is bound by the four DFMA of
// each term's complex multiply-add.  In double-float a term costs ~48 fp32
// operations, which leaves the kernel bound by its integer work and gathers.
// Accuracy: the split of phi, of the phases and of the couplings, and the
// dropped lo*lo products each contribute a few 2^-48 relative per term; a
// row of ~30 terms stays within ~1e-14 of the exact product (relative to the
// row's largest term).  The solvers apply H this way to the double-float copy
// of each Lanczos vector they already keep.
#include "qs3_df.cuh"
#include "qs3_hphi_common.cuh"

namespace qs3 {

struct dfc { dfl re, im; };

// complex double-float p times a real double-float f
__device__ __forceinline__ float4 dfc_scale(float4 p, dfl f) {
    const dfl r = df_mul({p.x, p.y}, f), i = df_mul({p.z, p.w}, f);
    return make_float4(r.hi, r.lo, i.hi, i.lo);
}
// acc += p x for complex double-float p, x
__device__ __forceinline__ void dfc_mac(dfc &acc, float4 p, float4 x) {
    df_mac(acc.re, p.x, p.y, x.x, x.y);
    df_mac(acc.re, -p.z, -p.w, x.z, x.w);
    df_mac(acc.im, p.x, p.y, x.z, x.w);
    df_mac(acc.im, p.z, p.w, x.x, x.y);
}
__device__ __forceinline__ double2 dfc_out(const dfc &a) {
    return make_double2((double)a.re.hi + (double)a.re.lo, (double)a.im.hi + (double)a.im.lo);
}

// one thread per row, persistent grid over the tiles of all sectors (the
// structure of k_hphi); phi may be phi + (*dx) ld when dx is given (a vector
// of a stored set chosen by an index in device memory, as inside a captured
// CUDA graph).  ODF:
// psi is written in double-float form too (float4, renormalised), else as
// complex128.  DEGB > 0 (representative table only): per occupied site the
// first DEGB hops go in stages -- all target ranks, then all table entries,
// then all rows, then all gathers -- so each stage's independent loads are in
// flight together instead of one dependent chain per hop.
template <int ND, bool TB, bool ODF, int DEGB>
__global__ void __launch_bounds__(NTHREADS, DEGB == 4 ? 4 : 3) k_hphi_df(LatView L, const SecView *__restrict__ secs,
                                                      const int *__restrict__ tile0, int S, int ntiles,
                                                      const float4 *__restrict__ phi, void *__restrict__ psi,
                                                      const int *__restrict__ active, const int *__restrict__ dx,
                                                      uint64_t ld) {
    extern __shared__ __align__(16) unsigned char smem[];
    SmemLayout sm = carve(L, smem);
    stage_tables(L, sm.sC, sm.sxyz);
    // sqrt(a / b) for |Stab| values a, b <= 8 (|Stab| divides N_down <= 8:
    // a translation fixing a state permutes its down spins without fixed points)
    __shared__ float2 srt[81];
    if (threadIdx.x < 81) {
        const int a = threadIdx.x / 9, b = threadIdx.x % 9;
        srt[threadIdx.x] = split_d(b ? sqrt((double)a / (double)b) : 0.0);
    }
    if (dx) phi += (uint64_t)(*dx) * ld;
    const float2 jsp = split_d(L.jh_uniform);
    const dfl juni = {jsp.x, jsp.y};
    const bool uni = L.jh_uniform != 0.0;
    __syncthreads();
    float4 *ph = (float4 *)sm.sph;     // the sector's phases in double-float
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s = (S == 1) ? 0 : sector_of_tile(tile0, S, t);
        if (active && !active[s]) continue;
        const SecView sv = secs[s];
        if (s != cur) {
            __syncthreads();
            for (int i = threadIdx.x; i < L.N; i += blockDim.x) ph[i] = sv.phdf[i];
            __syncthreads();
            cur = s;
        }
        const uint64_t row = (uint64_t)(t - sv.tile0) * TILE + threadIdx.x;
        if (row >= sv.dim) continue;
        const uint64_t rank = __ldg(sv.sigma + row);
        int c[ND];
        unrank(rank, sm.sC, L.np1, c);
        const float4 *ph_in = phi + sv.off;
        const int st_row = sv.stab[row];
        dfl e = {L.c0f, L.c0lo}, dd = {0.f, 0.f};
        // the hop terms: phase x phi (uniform J^xy, multiplied in once at the
        // end) or coupling x phase x phi
        dfc acch = {{0.f, 0.f}, {0.f, 0.f}};
        // one hop's term: bond q, target translation u, |Stab| st, phi at the target
        auto add_hop = [&](int q, int u, int st, float4 xv) {
            float4 p = ph[u];
            if (uni) {
                // uniform J^xy: the amplitude multiplies the row's hop sum once
                if (st != st_row) {
                    const float2 r = srt[st * 9 + st_row];
                    p = dfc_scale(p, {r.x, r.y});
                }
                dfc_mac(acch, p, xv);
            } else {
                dfl w = {__ldg(L.adj_jxy_f + q), __ldg(L.adj_jxy_lo + q)};
                if (st != st_row) {
                    const float2 r = srt[st * 9 + st_row];
                    w = df_mul(w, {r.x, r.y});
                }
                dfc_mac(acch, dfc_scale(p, w), xv);
            }
        };
#pragma unroll 1
        for (int m = 0; m < ND; ++m) {
            const int i = pick(c, m);
            e = df_sum(e, {__ldg(L.u_f + i), __ldg(L.u_lo + i)});
            const int e0 = __ldg(L.adj_ptr + i), e1 = __ldg(L.adj_ptr + i + 1);
            int qs = e0;
            if constexpr (TB && DEGB > 0) {
                // neighbours of c_m in the sorted list: j keeps position m when
                // lo < j < hi, and then only the m-th term of the rank changes
                const int lo = m > 0 ? pick(c, m - 1) : -1, hi = m < ND - 1 ? pick(c, m + 1) : L.N;
                const uint64_t rank_m = rank - sm.sC[(m + 1) * L.np1 + i];
                uint32_t key[DEGB];
#pragma unroll
                for (int b = 0; b < DEGB; ++b) {
                    const int q = e0 + b;
                    key[b] = 0xffffffffu;
                    if (q < e1) {
                        const int j = __ldg(L.adj_nbr + q);
                        bool occ = false;
#pragma unroll
                        for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                        if (occ) {
                            dd = df_sum(dd, {__ldg(L.adj_jz_f + q), __ldg(L.adj_jz_lo + q)});
                        } else if (j > lo && j < hi) {
                            key[b] = (uint32_t)(rank_m + sm.sC[(m + 1) * L.np1 + j]);   // table ranks are below 2^32
                        } else {
                            int tt[ND];
#pragma unroll
                            for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                            sort_net(tt);
                            key[b] = (uint32_t)rank_of(tt, sm.sC, L.np1);
                        }
                    }
                }
#pragma unroll
                for (int b = 0; b < DEGB; ++b)
                    if (key[b] != 0xffffffffu) key[b] = __ldg(L.orb + key[b]);
                int32_t row2[DEGB];
#pragma unroll
                for (int b = 0; b < DEGB; ++b)
                    row2[b] = (key[b] != 0xffffffffu && (key[b] >> 12) < L.n_orb) ? __ldg(sv.t2 + (key[b] >> 12)) : -1;
                float4 xv[DEGB];
                int stv[DEGB];
#pragma unroll
                for (int b = 0; b < DEGB; ++b)
                    if (row2[b] >= 0) {
                        xv[b] = ph_in[row2[b]];
                        stv[b] = __ldg(sv.stab + row2[b]);
                    }
#pragma unroll
                for (int b = 0; b < DEGB; ++b)
                    if (row2[b] >= 0) add_hop(e0 + b, (int)(key[b] & 4095u), stv[b], xv[b]);
                qs = e0 + DEGB;
            }
            for (int q = qs; q < e1; ++q) {
                const int j = __ldg(L.adj_nbr + q);
                bool occ = false;
#pragma unroll
                for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                if (occ) {
                    dd = df_sum(dd, {__ldg(L.adj_jz_f + q), __ldg(L.adj_jz_lo + q)});
                    continue;
                }
                int tt[ND];
#pragma unroll
                for (int k = 0; k < ND; ++k) tt[k] = (k == m) ? j : c[k];
                uint32_t idx;
                int u;
                if constexpr (TB) {
                    sort_net(tt);
                    const uint32_t ent = __ldg(L.orb + rank_of(tt, sm.sC, L.np1));
                    if ((ent >> 12) >= L.n_orb) continue;     // never for a complete table
                    const int32_t row2 = __ldg(sv.t2 + (ent >> 12));
                    if (row2 < 0) continue;
                    idx = (uint32_t)row2;
                    u = (int)(ent & 4095u);
                } else {
                    int rep[ND];
                    int ax, by, cz;
                    const uint64_t r2 = canon(tt, L, sm.sxyz, sm.sC, rep, ax, by, cz);
                    if (!sigma_find(sv, prefix_of(rep, sm.sC, L.np1), r2, idx)) continue;
                    u = ax + L.L[0] * (by + L.L[1] * cz);
                }
                add_hop(q, u, __ldg(sv.stab + idx), ph_in[idx]);
            }
        }
        dfc acc = acch;
        if (uni) {
            const dfl hr = df_norm(acch.re), hi = df_norm(acch.im);
            acc = {{0.f, 0.f}, {0.f, 0.f}};
            df_mac(acc.re, juni.hi, juni.lo, hr.hi, hr.lo);
            df_mac(acc.im, juni.hi, juni.lo, hi.hi, hi.lo);
        }
        const float4 x0 = ph_in[row];
        e = df_sum(e, {0.5f * dd.hi, 0.5f * dd.lo});
        df_mac(acc.re, e.hi, e.lo, x0.x, x0.y);
        df_mac(acc.im, e.hi, e.lo, x0.z, x0.w);
        if constexpr (ODF) {
            const dfl re = df_norm(acc.re), im = df_norm(acc.im);
            ((float4 *)psi)[sv.off + row] = make_float4(re.hi, re.lo, im.hi, im.lo);
        } else {
            ((double2 *)psi)[sv.off + row] = dfc_out(acc);
        }
    }
}

// N_down = 0: the single all-up state, H = c0
__global__ void k_diag0_df(double c0, uint64_t n, const float4 *__restrict__ phi, double2 *__restrict__ psi) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 v = phi[i];
        psi[i] = make_double2(c0 * ((double)v.x + (double)v.y), c0 * ((double)v.z + (double)v.w));
    }
}

__global__ void k_split_df(const double2 *__restrict__ x, float4 *__restrict__ y, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        y[i] = split2(x[i]);
}

template <int ND, bool TB, bool ODF, int DEGB>
static int hphi_df_ndt(Basis &B, const float4 *phi, const int *dx, uint64_t ld, void *psi, cudaStream_t st,
                       const int *active) {
    static std::atomic<unsigned long long> cache{0};
    int grid = 1, occ = 1;
    QS3_TRY(launch_rows(k_hphi_df<ND, TB, ODF, DEGB>, B, B.smem_bytes, cache, &grid, &occ));
    if (B.ntiles == 0) return QS3_OK;
    auto launch = [&](int g) {
        k_hphi_df<ND, TB, ODF, DEGB><<<g, NTHREADS, B.smem_bytes, st>>>(B.lv, B.d_secs.as<SecView>(),
                                                                          B.d_tile0.as<int>(), B.S, B.ntiles, phi, psi,
                                                                          active, dx, ld);
    };
    int &bps = B.tune_hphi[QS3_C128DF];
    if (bps == 0) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        QS3_CUDA(cudaStreamIsCapturing(st, &cst));
        if (cst == cudaStreamCaptureStatusNone) {
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
static int hphi_df_nd(Basis &B, const float4 *phi, const int *dx, uint64_t ld, void *psi, bool out_df,
                      cudaStream_t st, const int *active) {
    // table: hops staged DEGB = 4 (square, chain) or 6 (cubic, triangular) at a time
    if (B.lv.orb) {
        if (B.max_degree <= 4)
            return out_df ? hphi_df_ndt<ND, true, true, 4>(B, phi, dx, ld, psi, st, active)
                          : hphi_df_ndt<ND, true, false, 4>(B, phi, dx, ld, psi, st, active);
        return out_df ? hphi_df_ndt<ND, true, true, 6>(B, phi, dx, ld, psi, st, active)
                      : hphi_df_ndt<ND, true, false, 6>(B, phi, dx, ld, psi, st, active);
    }
    return out_df ? hphi_df_ndt<ND, false, true, 0>(B, phi, dx, ld, psi, st, active)
                  : hphi_df_ndt<ND, false, false, 0>(B, phi, dx, ld, psi, st, active);
}

int hphi_df_launch(Basis &B, const void *phi, const int *dx, uint64_t ld, void *psi, cudaStream_t st,
                   const int *active, bool out_df) {
    if (!phi || !psi) return set_err(QS3_ERR_INVALID_ARG, "NULL vector");
    if (phi == psi) return set_err(QS3_ERR_INVALID_ARG, "phi and psi alias");
    if (!B.has_k) return set_err(QS3_ERR_STATE, "C128DF needs a basis with momentum sectors");
    if (B.total == 0) return QS3_OK;
    const float4 *p = (const float4 *)phi;
    void *q = psi;
    if (B.nd == 0) {
        if (dx || out_df) return set_err(QS3_ERR_INVALID_ARG, "double-float output or device index needs N_down > 0");
        const int grid = (int)std::min<uint64_t>((B.total + 255) / 256, 1024);
        k_diag0_df<<<grid, 256, 0, st>>>(B.lv.c0, B.total, p, (double2 *)q);
        QS3_LAUNCHED();
        return QS3_OK;
    }
    switch (B.nd) {
        case 1: return hphi_df_nd<1>(B, p, dx, ld, q, out_df, st, active);
        case 2: return hphi_df_nd<2>(B, p, dx, ld, q, out_df, st, active);
        case 3: return hphi_df_nd<3>(B, p, dx, ld, q, out_df, st, active);
        case 4: return hphi_df_nd<4>(B, p, dx, ld, q, out_df, st, active);
        case 5: return hphi_df_nd<5>(B, p, dx, ld, q, out_df, st, active);
        case 6: return hphi_df_nd<6>(B, p, dx, ld, q, out_df, st, active);
        case 7: return hphi_df_nd<7>(B, p, dx, ld, q, out_df, st, active);
        case 8: return hphi_df_nd<8>(B, p, dx, ld, q, out_df, st, active);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

}  // namespace qs3

using namespace qs3;

extern "C" int qs3_split_df(const void *x, void *x_df, uint64_t n, void *stream) {
    clear_err();
    if (n == 0) return QS3_OK;
    if (!x || !x_df) return set_err(QS3_ERR_INVALID_ARG, "NULL vector");
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, 4096);
    k_split_df<<<grid, 256, 0, (cudaStream_t)stream>>>((const double2 *)x, (float4 *)x_df, n);
    QS3_LAUNCHED();
    return QS3_OK;
}
