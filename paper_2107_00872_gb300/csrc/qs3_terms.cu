// qs3_terms.cu -- stored-term H Phi for k-sector bases (an opt-in variant of
// the matrix-free product of Alg. 9, which the paper recomputes every time).
//
// Every off-diagonal term of Alg. 9 that lands on a member of the sector is
// enumerated once, in the order the on-the-fly kernel visits them (down spin
// m, then bond q of its site), and kept as
//     col  = the target's row in the sector (uint32),
//     code = u | st << 12 | q << 16
// with u the translation to the target's representative (its phase index),
// st the target's |Stab| and q the bond's adjacency entry (its amplitude),
// plus the diagonal of every row (fp64).  Row pointers come from an
// exclusive scan of the per-row term counts (a library scan).  A later H Phi
// is then a gather SpMV that recomputes only the coefficient from the code,
// in the same arithmetic order as the matrix-free kernel: complex128 results
// are identical bit for bit; complex64 rounds the stored fp64 diagonal once.
// Memory: 8 bytes per term + 16 bytes per row.
#include <algorithm>
#include <string>

#include <cub/cub.cuh>

#include "qs3_hphi_common.cuh"

namespace qs3 {

// FILL = false: cnt[g] = number of terms of global row g;
// FILL = true:  col/code from rptr[g], diag[g]
template <int ND, bool TB, bool FILL>
__global__ void __launch_bounds__(NTHREADS) k_terms(LatView L, const SecView *__restrict__ secs,
                                                    const int *__restrict__ tile0, int S, int ntiles,
                                                    uint64_t *__restrict__ cnt, const uint64_t *__restrict__ rptr,
                                                    uint32_t *__restrict__ col, uint32_t *__restrict__ code,
                                                    double *__restrict__ diag) {
    extern __shared__ __align__(16) unsigned char smem[];
    SmemLayout sm = carve(L, smem);
    stage_tables(L, sm.sC, sm.sxyz);
    __syncthreads();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s = (S == 1) ? 0 : sector_of_tile(tile0, S, t);
        const SecView sv = secs[s];
        const uint64_t row = (uint64_t)(t - sv.tile0) * TILE + threadIdx.x;
        if (row >= sv.dim) continue;
        const uint64_t g = sv.off + row;
        int c[ND];
        unrank(__ldg(sv.sigma + row), sm.sC, L.np1, c);
        double e = L.c0, dd = 0.0;
        uint64_t w = FILL ? rptr[g] : 0;
        for (int m = 0; m < ND; ++m) {
            const int i = pick(c, m);
            e += __ldg(L.u + i);
            const int e0 = __ldg(L.adj_ptr + i), e1 = __ldg(L.adj_ptr + i + 1);
            for (int q = e0; q < e1; ++q) {
                const int j = __ldg(L.adj_nbr + q);
                bool occ = false;
#pragma unroll
                for (int k = 0; k < ND; ++k) occ |= (c[k] == j);
                if (occ) {
                    dd += __ldg(L.adj_jz + q);
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
                    if ((ent >> 12) >= L.n_orb) continue;
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
                if constexpr (FILL) {
                    const uint32_t st = __ldg(sv.stab + idx);
                    col[w] = idx;
                    code[w] = (uint32_t)u | (st << 12) | ((uint32_t)q << 16);
                }
                ++w;
            }
        }
        if constexpr (FILL) diag[g] = e + 0.5 * dd;
        else cnt[g] = w;
    }
}

// psi = H phi from the stored terms (same coefficient arithmetic and order as
// the matrix-free k_hphi<ND, VT, true, *>)
template <typename VT>
__global__ void __launch_bounds__(NTHREADS, 4) k_hphi_st(LatView L, const SecView *__restrict__ secs,
                                                       const int *__restrict__ tile0, int S, int ntiles,
                                                       const uint64_t *__restrict__ rptr,
                                                       const uint32_t *__restrict__ col,
                                                       const uint32_t *__restrict__ code,
                                                       const double *__restrict__ diag, const VT *__restrict__ phi,
                                                       VT *__restrict__ psi, const int *__restrict__ active) {
    using R = typename VTr<VT>::R;
    using CT = typename VTr<VT>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    R *snorm = (R *)smem;                          // [0..8] sqrt(s), [9..17] 1/sqrt(s)
    CT *ph = (CT *)(smem + 16 * 18);               // the current sector's phases
    if (threadIdx.x < 9) {
        snorm[threadIdx.x] = (R)sqrt((double)threadIdx.x);
        snorm[9 + threadIdx.x] = threadIdx.x ? (R)(1.0 / sqrt((double)threadIdx.x)) : (R)0;
    }
    const R *jxy = jxy_table<VT>(L);
    const R juni = (R)L.jh_uniform;
    const bool uni = juni != (R)0;
    __syncthreads();
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s = (S == 1) ? 0 : sector_of_tile(tile0, S, t);
        if (active && !active[s]) continue;
        const SecView sv = secs[s];
        if (s != cur) {
            __syncthreads();
            const CT *gph = phase_table<CT>(sv);
            for (int i = threadIdx.x; i < L.N; i += blockDim.x) ph[i] = gph[i];
            __syncthreads();
            cur = s;
        }
        const uint64_t row = (uint64_t)(t - sv.tile0) * TILE + threadIdx.x;
        if (row >= sv.dim) continue;
        const uint64_t g = sv.off + row;
        const VT *ph_in = phi + sv.off;
        const VT x0 = ph_in[row];
        const int st_row = sv.stab[row];
        const R rs = snorm[9 + st_row];
        CT acc, acch;
        acc.x = 0; acc.y = 0;
        acch.x = 0; acch.y = 0;
        const uint64_t t1 = rptr[g + 1];
        // one term: coefficient from its code, accumulated in list order
        auto term = [&](uint32_t cd, VT x) {
            CT p = ph[cd & 4095u];
            const int st = (int)((cd >> 12) & 15u);
            if (uni) {
                if (st != st_row) {
                    const R f = snorm[st] * rs;
                    p.x *= f;
                    p.y *= f;
                }
                acc_add(acch, p, x);
            } else {
                const R jh = __ldg(jxy + (cd >> 16));
                const R w = (st == st_row) ? jh : jh * snorm[st] * rs;
                p.x *= w;
                p.y *= w;
                acc_add(acc, p, x);
            }
        };
        // groups of four terms: their index loads and gathers are in flight
        // together, the sums still run in list order
        uint64_t tt = rptr[g];
        for (; tt + 4 <= t1; tt += 4) {
            uint32_t cd[4], ix[4];
            VT v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cd[j] = __ldg(code + tt + j);
                ix[j] = __ldg(col + tt + j);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = ph_in[ix[j]];
#pragma unroll
            for (int j = 0; j < 4; ++j) term(cd[j], v[j]);
        }
        for (; tt < t1; ++tt) term(__ldg(code + tt), ph_in[__ldg(col + tt)]);
        if (uni) madd_r(acc, juni, acch);
        madd_r(acc, (R)diag[g], x0);
        store(psi + sv.off + row, acc);
    }
}

static int grid_tiles(const Basis &B, int per_sm) {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(B.ntiles, nsm * per_sm));
}

template <int ND>
static int build_terms_nd(Basis &B, size_t max_bytes) {
    uint64_t nz = 0;
    QS3_TRY(count_nnz(B, &nz));
    const uint64_t nterm = nz - B.total;
    const uint64_t bytes = nterm * 8 + (B.total + 1) * 8 + B.total * 8;
    if (bytes > max_bytes)
        return set_err(QS3_ERR_OOM, "stored terms need %llu bytes, above the limit", (unsigned long long)bytes);
    if (nterm >= (1ull << 40)) return set_err(QS3_ERR_OVERFLOW, "too many terms");
    DevBuf cnt, rptr, col, code, dg;
    QS3_TRY(cnt.alloc((B.total + 1) * 8));
    QS3_TRY(rptr.alloc((B.total + 1) * 8));
    QS3_CUDA(cudaMemset(cnt.p, 0, (B.total + 1) * 8));
    const bool tb = B.lv.orb != nullptr;
    const int grid = grid_tiles(B, 8);
    if (tb) {
        QS3_CUDA(cudaFuncSetAttribute(k_terms<ND, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_terms<ND, true, false><<<grid, NTHREADS, B.smem_bytes>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(),
                                                                   B.S, B.ntiles, cnt.as<uint64_t>(), nullptr,
                                                                   nullptr, nullptr, nullptr);
    } else {
        QS3_CUDA(cudaFuncSetAttribute(k_terms<ND, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_terms<ND, false, false><<<grid, NTHREADS, B.smem_bytes>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(),
                                                                    B.S, B.ntiles, cnt.as<uint64_t>(), nullptr,
                                                                    nullptr, nullptr, nullptr);
    }
    QS3_LAUNCHED();
    size_t tb_bytes = 0;
    QS3_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb_bytes, cnt.as<uint64_t>(), rptr.as<uint64_t>(),
                                           (int64_t)(B.total + 1)));
    DevBuf tmp;
    QS3_TRY(tmp.alloc(tb_bytes));
    QS3_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, tb_bytes, cnt.as<uint64_t>(), rptr.as<uint64_t>(),
                                           (int64_t)(B.total + 1)));
    uint64_t last = 0;
    QS3_CUDA(cudaMemcpy(&last, rptr.as<uint64_t>() + B.total, 8, cudaMemcpyDeviceToHost));
    if (last != nterm)
        return set_err(QS3_ERR_STATE, "stored terms: %llu counted, %llu expected", (unsigned long long)last,
                       (unsigned long long)nterm);
    cnt.release();
    tmp.release();
    QS3_TRY(col.alloc(nterm * 4));
    QS3_TRY(code.alloc(nterm * 4));
    QS3_TRY(dg.alloc(B.total * 8));
    if (tb) {
        QS3_CUDA(cudaFuncSetAttribute(k_terms<ND, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_terms<ND, true, true><<<grid, NTHREADS, B.smem_bytes>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(),
                                                                  B.S, B.ntiles, nullptr, rptr.as<uint64_t>(),
                                                                  col.as<uint32_t>(), code.as<uint32_t>(),
                                                                  dg.as<double>());
    } else {
        QS3_CUDA(cudaFuncSetAttribute(k_terms<ND, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        k_terms<ND, false, true><<<grid, NTHREADS, B.smem_bytes>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(),
                                                                   B.S, B.ntiles, nullptr, rptr.as<uint64_t>(),
                                                                   col.as<uint32_t>(), code.as<uint32_t>(),
                                                                   dg.as<double>());
    }
    QS3_LAUNCHED();
    QS3_CUDA(cudaDeviceSynchronize());
    B.d_trp = std::move(rptr);
    B.d_tcol = std::move(col);
    B.d_tcode = std::move(code);
    B.d_tdiag = std::move(dg);
    B.n_terms = nterm;
    B.stored_terms = true;
    return QS3_OK;
}

int build_terms(Basis &B, size_t max_bytes) {
    if (!B.has_k || B.nd == 0 || B.total == 0) return set_err(QS3_ERR_STATE, "stored terms serve k-sector bases only");
    if (B.N > 4096) return set_err(QS3_ERR_OVERFLOW, "N > 4096");
    if (2 * (size_t)B.nb >= 65536) return set_err(QS3_ERR_OVERFLOW, "more than 32767 bonds");
    if (B.stored_terms) return QS3_OK;
    switch (B.nd) {
        case 1: return build_terms_nd<1>(B, max_bytes);
        case 2: return build_terms_nd<2>(B, max_bytes);
        case 3: return build_terms_nd<3>(B, max_bytes);
        case 4: return build_terms_nd<4>(B, max_bytes);
        case 5: return build_terms_nd<5>(B, max_bytes);
        case 6: return build_terms_nd<6>(B, max_bytes);
        case 7: return build_terms_nd<7>(B, max_bytes);
        case 8: return build_terms_nd<8>(B, max_bytes);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

void drop_terms(Basis &B) {
    B.stored_terms = false;
    B.d_trp.release();
    B.d_tcol.release();
    B.d_tcode.release();
    B.d_tdiag.release();
    B.n_terms = 0;
}

template <typename VT>
static int hphi_st_vt(Basis &B, const void *phi, void *psi, cudaStream_t st, const int *active) {
    using CT = typename VTr<VT>::C;
    const size_t smem = 16 * 18 + (size_t)B.N * sizeof(CT);
    const int grid = grid_tiles(B, 8);
    k_hphi_st<VT><<<grid, NTHREADS, smem, st>>>(B.lv, B.d_secs.as<SecView>(), B.d_tile0.as<int>(), B.S, B.ntiles,
                                                 B.d_trp.as<uint64_t>(), B.d_tcol.as<uint32_t>(),
                                                 B.d_tcode.as<uint32_t>(), B.d_tdiag.as<double>(), (const VT *)phi,
                                                 (VT *)psi, active);
    QS3_LAUNCHED();
    return QS3_OK;
}

int hphi_stored_launch(Basis &B, qs3_dtype dt, const void *phi, void *psi, cudaStream_t st, const int *active) {
    if (B.ntiles == 0) return QS3_OK;
    if (dt == QS3_C128) return hphi_st_vt<double2>(B, phi, psi, st, active);
    if (dt == QS3_C64) return hphi_st_vt<float2>(B, phi, psi, st, active);
    return set_err(QS3_ERR_STATE, "k-sector bases need complex vectors (C64/C128)");
}

}  // namespace qs3

using namespace qs3;

extern "C" int qs3_basis_store_terms(qs3_basis_t b, int32_t mode, uint64_t *bytes) {
    clear_err();
    if (!b) return set_err(QS3_ERR_INVALID_ARG, "basis is NULL");
    if (mode < -1 || mode > 1) return set_err(QS3_ERR_INVALID_ARG, "mode %d", mode);
    int st = QS3_OK;
    if (mode == 0) {
        drop_terms(b->B);
    } else if (mode == 1) {
        size_t fr = 0, tt = 0;
        QS3_CUDA(cudaMemGetInfo(&fr, &tt));
        st = build_terms(b->B, fr / 2);
        if (st != QS3_OK) {
            std::string msg = last_err();
            drop_terms(b->B);
            set_err(st, "%s", msg.c_str());
        }
    }
    const Basis &B = b->B;
    if (bytes) *bytes = B.stored_terms ? B.n_terms * 8 + (B.total + 1) * 8 + B.total * 8 : 0;
    return st;
}
