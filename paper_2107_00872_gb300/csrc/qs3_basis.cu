// qs3_basis.cu -- lattice ingest and symmetry-adapted basis construction on
// the device (Sec. "Representative states and Hamiltonian matrix elements in
// symmetry-adapted basis sets", Alg. 5-6 of the paper, re-designed).
//
// Instead of testing all C(N, N_down) states with all N translations
// (Alg. 5/6), the device enumerates the C(N-1, N_down-1) states that have a
// down spin at site 0.  Every translation orbit contains such states: the
// translates T^{-pos(c_m)} c that move one of its spins to the origin.  A
// state c emits its orbit's representative exactly once, when c has the
// smallest rank among those origin-containing translates.  The stabiliser
// of c is the set of pos(c_m) whose translate reproduces c, which gives
// |Stab| and the compatibility test e^{ik.t} = 1 on it (N_{a,k} > 0 in
// Alg. 5).  The representatives are sorted by rank (CUB radix sort, a
// library primitive) and indexed by a prefix table over their two largest
// sites.
#include <cub/cub.cuh>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>

#include "qs3_internal.cuh"
#include "qs3_fixed.cuh"

namespace qs3 {

// ------------------------------------------------------------ error state
static thread_local char g_err[1024];

int set_err(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_err() { g_err[0] = 0; }

static std::atomic<unsigned long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

const char *last_err() { return g_err; }

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
}

// allocation fault injection (qs3_inject_alloc_failure): the number of
// allocations still allowed to succeed, or -1 when off
static std::atomic<long long> g_alloc_budget{-1};
static std::atomic<int> g_wait_starve{0};
int take_wait_injection() {
    for (int n = g_wait_starve.load(); n > 0;)
        if (g_wait_starve.compare_exchange_weak(n, n - 1)) return 1;
    return 0;
}

int DevBuf::alloc(size_t bytes) {
    release();
    if (bytes == 0) bytes = 16;
    for (long long b = g_alloc_budget.load(); b >= 0;) {
        if (b == 0) return set_err(QS3_ERR_OOM, "device allocation of %zu bytes refused (injected failure)", bytes);
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return set_err(e == cudaErrorMemoryAllocation ? QS3_ERR_OOM : QS3_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                       cudaGetErrorString(e));
    }
    n = bytes;
    return QS3_OK;
}

int DevBuf::upload(const void *src, size_t bytes) {
    QS3_TRY(alloc(bytes));
    if (bytes) QS3_CUDA(cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice));
    return QS3_OK;
}

// must match carve() in qs3_hphi.cu: binomial rows 0..nd+2, coordinates (k
// only), sqrt table (18 doubles), the current sector's phases (k only)
size_t row_kernel_smem(const Basis &B, int /*extra_nd*/) {
    size_t s = (size_t)(B.nd + 3) * (B.N + 1) * sizeof(uint64_t);
    if (B.has_k) s += (size_t)B.N * sizeof(uint32_t);
    s = (s + 15) & ~(size_t)15;
    s += 18 * sizeof(double);
    s = (s + 15) & ~(size_t)15;
    if (B.has_k) s += (size_t)B.N * 2 * sizeof(double);
    return s;
}

// ------------------------------------------------------ enumeration kernel

// Candidates: the states with a spin at site (cell 0, place s0) and none on
// places below s0 (s0 = the lowest place of the cell that the state
// occupies; with one spin per cell s0 = 0): the other N_down - 1 spins are
// an (N_down - 1)-subset of the M - 1 sites after it in the list of sites
// with place >= s0 (index q -> place s0 + q % w, cell q / w, w = nsub - s0).
// Every orbit has such members (move any spin on place s0 to cell 0); a
// candidate is designated when it has the smallest rank of them, so each
// orbit is taken once, from its designated member, with |Stab| (the moves
// that give the candidate back) and the compatibility of those moves with K.
template <int ND>
__global__ void __launch_bounds__(NTHREADS) k_enum_reps(LatView L, int Kx, int Ky, int Kz, int s0, uint64_t ncand,
                                                        int emit, unsigned long long *counter,
                                                        uint64_t *out_rank, uint8_t *out_stab) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sC = (uint64_t *)smem;
    uint32_t *sxyz = (uint32_t *)(sC + (L.nd + 3) * L.np1);
    const int nC = (L.nd + 3) * L.np1;
    for (int i = threadIdx.x; i < nC; i += blockDim.x) sC[i] = L.binom[i];
    for (int i = threadIdx.x; i < L.N; i += blockDim.x) sxyz[i] = L.xyz[i];
    __syncthreads();
    const int Lx = L.L[0], Ly = L.L[1], Lz = L.L[2];
    const int G = L.ncell, ns = L.nsub, w = ns - s0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < ncand; base += stride) {
        const uint64_t j = base + threadIdx.x;
        bool take = false;
        uint64_t rep_rank = 0;
        int st = 0;
        if (j < ncand) {
            int c[ND];
            c[0] = s0;
            if (ND >= 2) {
                constexpr int NM1 = (ND > 1) ? ND - 1 : 1;
                int cc[NM1];
                unrank<NM1>(j, sC, L.np1, cc);
#pragma unroll
                for (int m = 0; m + 1 < ND; ++m) {
                    const int q = cc[m] + 1;
                    c[m + 1] = (w == 1) ? s0 + ns * q : s0 + q % w + ns * (q / w);
                }
            }
            const uint64_t rc = rank_of(c, sC, L.np1);
            int X[ND], Y[ND], Z[ND], SB[ND];
#pragma unroll
            for (int m = 0; m < ND; ++m) {
                uint32_t p = sxyz[c[m]];
                X[m] = p & 2047u;
                Y[m] = (p >> 11) & 2047u;
                Z[m] = p >> 22;
                SB[m] = ns > 1 ? c[m] % ns : 0;
            }
            bool designated = true, compat = true;
#pragma unroll
            for (int m = 0; m < ND; ++m) {
                if (SB[m] != s0) continue;
                int sl[ND];
#pragma unroll
                for (int q = 0; q < ND; ++q) {
                    int xx = X[q] - X[m]; xx += (xx < 0) ? Lx : 0;
                    int yy = Y[q] - Y[m]; yy += (yy < 0) ? Ly : 0;
                    int zz = Z[q] - Z[m]; zz += (zz < 0) ? Lz : 0;
                    sl[q] = SB[q] + ns * (xx + Lx * (yy + Ly * zz));
                }
                sort_net(sl);
                const uint64_t rm = rank_of(sl, sC, L.np1);
                designated &= (rm >= rc);
                if (rm == rc) {
                    ++st;
                    // stabiliser element t = cell(c_m): compatible iff k.t is a multiple of 2 pi
                    long long num = (long long)Kx * X[m] * (G / Lx) + (long long)Ky * Y[m] * (G / Ly) +
                                    (long long)Kz * Z[m] * (G / Lz);
                    compat &= (num % G) == 0;
                }
            }
            take = designated && compat;
            if (take && emit) {
                int rep[ND];
                int ax, by, cz;
                rep_rank = canon(c, L, sxyz, sC, rep, ax, by, cz);
            }
        }
        // warp-aggregated slot allocation
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        const int lane = threadIdx.x & 31;
        unsigned long long basepos = 0;
        if (lane == 0 && mask) basepos = atomicAdd(counter, (unsigned long long)__popc(mask));
        basepos = __shfl_sync(0xffffffffu, basepos, 0);
        if (take && emit) {
            const unsigned long long pos = basepos + __popc(mask & ((1u << lane) - 1u));
            out_rank[pos] = rep_rank;
            out_stab[pos] = (uint8_t)st;
        }
    }
}

template <int ND>
__global__ void k_prefix(LatView L, const uint64_t *__restrict__ sigma, uint64_t d, uint32_t *__restrict__ P) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sC = (uint64_t *)smem;
    const int nC = (L.nd + 3) * L.np1;
    for (int i = threadIdx.x; i < nC; i += blockDim.x) sC[i] = L.binom[i];
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (uint64_t)gridDim.x * blockDim.x) {
        int c[ND];
        unrank(sigma[i], sC, L.np1, c);
        P[i] = prefix_of(c, sC, L.np1);
    }
}

// pidx[p] = first i with P[i] >= p, for p in [0, np]
__global__ void k_pidx(const uint32_t *__restrict__ P, uint64_t d, uint32_t np, uint32_t *__restrict__ pidx) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= np; p += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t lo = 0, hi = d;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if (P[mid] < p) lo = mid + 1; else hi = mid;
        }
        pidx[p] = (uint32_t)lo;
    }
}

// the representatives of momentum K (each orbit once, compatible ones only),
// sorted by rank0, with |Stab|: d of them in kout / vout
template <int ND>
static int enum_sorted_reps(Basis &B, const int *K, DevBuf &kout, DevBuf &vout, uint64_t &d,
                            std::vector<uint64_t> &hb, int &nsm) {
    // per lowest occupied place s0 of the cell: C(M - 1, ND - 1) candidates,
    // M = (cells) (nsub - s0); one spin per cell: C(N - 1, ND - 1)
    hb.resize((size_t)(B.nd + 3) * (B.N + 1));
    QS3_CUDA(cudaMemcpy(hb.data(), B.d_binom.p, hb.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    const size_t smem = (size_t)(B.nd + 3) * (B.N + 1) * 8 + (size_t)B.N * 4;
    QS3_CUDA(cudaFuncSetAttribute(k_enum_reps<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
    DevBuf cnt;
    QS3_TRY(cnt.alloc(sizeof(unsigned long long)));
    QS3_CUDA(cudaMemset(cnt.p, 0, sizeof(unsigned long long)));
    int dev = 0;
    QS3_CUDA(cudaGetDevice(&dev));
    QS3_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    std::vector<uint64_t> nc(B.nsub, 0);
    for (int s0 = 0; s0 < B.nsub; ++s0) {
        const uint64_t M = (uint64_t)B.ncell * (B.nsub - s0);
        nc[s0] = (M >= 1 && M - 1 >= (uint64_t)(ND - 1)) ? hb[(size_t)(ND - 1) * (B.N + 1) + (M - 1)] : 0;
    }
    auto run = [&](int emit, uint64_t *kp, uint8_t *vp) -> int {
        for (int s0 = 0; s0 < B.nsub; ++s0) {
            if (!nc[s0]) continue;
            const uint64_t want = (nc[s0] + NTHREADS - 1) / NTHREADS;
            const int grid = (int)std::min<uint64_t>(want ? want : 1, (uint64_t)nsm * 8);
            k_enum_reps<ND><<<grid, NTHREADS, smem>>>(B.lv, K[0], K[1], K[2], s0, nc[s0], emit,
                                                      cnt.as<unsigned long long>(), kp, vp);
            QS3_LAUNCHED();
        }
        return QS3_OK;
    };
    QS3_TRY(run(0, nullptr, nullptr));
    d = 0;
    QS3_CUDA(cudaMemcpy(&d, cnt.p, sizeof(d), cudaMemcpyDeviceToHost));
    if (d >= (1ull << 32)) return set_err(QS3_ERR_OVERFLOW, "sector dimension %llu exceeds 2^32", (unsigned long long)d);
    DevBuf kin, vin;
    QS3_TRY(kin.alloc(d * 8));
    QS3_TRY(vin.alloc(d));
    QS3_CUDA(cudaMemset(cnt.p, 0, sizeof(unsigned long long)));
    QS3_TRY(run(1, kin.as<uint64_t>(), vin.as<uint8_t>()));
    QS3_TRY(kout.alloc(d * 8));
    QS3_TRY(vout.alloc(d));
    if (d > 0) {
        size_t tb = 0;
        QS3_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, kin.as<unsigned long long>(),
                                                 kout.as<unsigned long long>(), vin.as<uint8_t>(),
                                                 vout.as<uint8_t>(), (int64_t)d));
        DevBuf tmp;
        QS3_TRY(tmp.alloc(tb));
        QS3_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tb, kin.as<unsigned long long>(),
                                                 kout.as<unsigned long long>(), vin.as<uint8_t>(),
                                                 vout.as<uint8_t>(), (int64_t)d));
    }
    return QS3_OK;
}

template <int ND>
static int build_reps_nd(Basis &B, int s) {
    const int *K = &B.K[3 * s];
    std::vector<uint64_t> hb;
    int nsm = 0;
    uint64_t d = 0;
    DevBuf kout, vout;
    QS3_TRY(enum_sorted_reps<ND>(B, K, kout, vout, d, hb, nsm));
    // prefix index
    const uint32_t np = (ND >= 2) ? (uint32_t)hb[2 * (size_t)(B.N + 1) + B.N] : (uint32_t)B.N;   // number of prefixes
    DevBuf P, pidx;
    QS3_TRY(P.alloc(d * 4));
    QS3_TRY(pidx.alloc(((size_t)np + 1) * 4));
    if (d > 0) {
        const size_t sm2 = (size_t)(B.nd + 3) * (B.N + 1) * 8;
        QS3_CUDA(cudaFuncSetAttribute(k_prefix<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
        int g2 = (int)std::min<uint64_t>((d + 255) / 256, (uint64_t)nsm * 8);
        k_prefix<ND><<<g2, 256, sm2>>>(B.lv, kout.as<uint64_t>(), d, P.as<uint32_t>());
        QS3_LAUNCHED();
    }
    int g3 = (int)std::min<uint64_t>((np + 256) / 256, (uint64_t)nsm * 8);
    k_pidx<<<g3, 256>>>(P.as<uint32_t>(), d, np, pidx.as<uint32_t>());
    QS3_LAUNCHED();
    QS3_CUDA(cudaDeviceSynchronize());
    B.dims[s] = d;
    B.d_sigma[s] = std::move(kout);
    B.d_stab[s] = std::move(vout);
    B.d_pidx[s] = std::move(pidx);
    return QS3_OK;
}

int build_sector_reps(Basis &B, int s) {
    switch (B.nd) {
        case 1: return build_reps_nd<1>(B, s);
        case 2: return build_reps_nd<2>(B, s);
        case 3: return build_reps_nd<3>(B, s);
        case 4: return build_reps_nd<4>(B, s);
        case 5: return build_reps_nd<5>(B, s);
        case 6: return build_reps_nd<6>(B, s);
        case 7: return build_reps_nd<7>(B, s);
        case 8: return build_reps_nd<8>(B, s);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

// ---------------------------------------------------- representative table
// For lattices whose C(N, N_down) states fit a 4-byte-per-state table, the
// result of the representative search of Alg. 7 for every state is tabulated
// once: orb[rank0(a)] = g << 12 | u with a = T_u (rep_g).  A hop target then
// costs one rank and two table loads instead of the search and the binary
// search in sigma.  It is the same function: where several translations reach
// the representative (a non-trivial stabiliser) they differ by a stabiliser
// element, whose phase is 1 on every sector that holds the representative.

// orb[rank0(T_u rep_g)] = g << 12 | u for every orbit g and translation u
template <int ND>
__global__ void __launch_bounds__(NTHREADS) k_orbit_fill(LatView L, const uint64_t *__restrict__ reps, uint64_t n,
                                                         uint32_t *__restrict__ orb) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sC = (uint64_t *)smem;
    uint32_t *sxyz = (uint32_t *)(sC + (L.nd + 3) * L.np1);
    const int nC = (L.nd + 3) * L.np1;
    for (int i = threadIdx.x; i < nC; i += blockDim.x) sC[i] = L.binom[i];
    for (int i = threadIdx.x; i < L.N; i += blockDim.x) sxyz[i] = L.xyz[i];
    __syncthreads();
    const int Lx = L.L[0], Ly = L.L[1], Lz = L.L[2], G = L.ncell, ns = L.nsub;
    const uint64_t total = n * (uint64_t)G;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t g = i / (uint64_t)G;
        const int u = (int)(i - g * (uint64_t)G);         // cell translation
        int c[ND];
        unrank(reps[g], sC, L.np1, c);
        const uint32_t pu = sxyz[u * ns];                  // the coordinates of cell u
        const int ux = pu & 2047u, uy = (pu >> 11) & 2047u, uz = pu >> 22;
        int t[ND];
#pragma unroll
        for (int m = 0; m < ND; ++m) {
            const uint32_t p = sxyz[c[m]];
            int x = (int)(p & 2047u) + ux, y = (int)((p >> 11) & 2047u) + uy, z = (int)(p >> 22) + uz;
            x -= (x >= Lx) ? Lx : 0;
            y -= (y >= Ly) ? Ly : 0;
            z -= (z >= Lz) ? Lz : 0;
            t[m] = c[m] % ns + ns * (x + Lx * (y + Ly * z));
        }
        sort_net(t);
        orb[rank_of(t, sC, L.np1)] = ((uint32_t)g << 12) | (uint32_t)u;
    }
}

// t2[s n + g] = row of representative g in sector s, -1 if the sector lacks it
__global__ void k_orbit_rows(const SecView *__restrict__ secs, int S, const uint64_t *__restrict__ reps, uint64_t n,
                             int32_t *__restrict__ t2) {
    const uint64_t total = n * (uint64_t)S;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i / n);
        const uint64_t g = i - (uint64_t)s * n;
        const uint64_t r = reps[g];
        const uint64_t *sig = secs[s].sigma;
        uint64_t lo = 0, hi = secs[s].dim;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (sig[mid] < r) lo = mid + 1; else hi = mid;
        }
        t2[i] = (lo < secs[s].dim && sig[lo] == r) ? (int32_t)lo : -1;
    }
}

// the per-site phases of every sector as fixed-point digits on the grid
// 2^-52 (re.P1, re.P0, im.P1, im.P0), for the integer H Phi
__global__ void k_phase_digits(const double2 *__restrict__ ph64, uint64_t n, int4 *__restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const double2 p = ph64[i];
        int a1, a0, b1, b0;
        fx_digits((uint32_t)__double2hiint(p.x), (uint32_t)__double2loint(p.x), 1023, a1, a0);
        fx_digits((uint32_t)__double2hiint(p.y), (uint32_t)__double2loint(p.y), 1023, b1, b0);
        out[i] = make_int4(a1, a0, b1, b0);
    }
}

template <int ND>
static int build_table_nd(Basis &B, size_t max_bytes) {
    std::vector<uint64_t> hb((size_t)(B.nd + 3) * (B.N + 1));
    QS3_CUDA(cudaMemcpy(hb.data(), B.d_binom.p, hb.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    const uint64_t ns = hb[(size_t)ND * (B.N + 1) + B.N];           // C(N, N_down)
    if (ns >= (1ull << 32)) return set_err(QS3_ERR_OVERFLOW, "C(N, N_down) = %llu states: no table", (unsigned long long)ns);
    const uint64_t n_est = ns / (uint64_t)B.ncell + 1;             // orbits, about C(N, N_down) / (cells)
    if (ns * 4 + n_est * 4 * (uint64_t)B.S > max_bytes)
        return set_err(QS3_ERR_OOM, "representative table of ~%llu bytes exceeds the limit",
                       (unsigned long long)(ns * 4 + n_est * 4 * (uint64_t)B.S));
    const int K0[3] = {0, 0, 0};                                   // every representative is compatible at k = 0
    DevBuf reps, stab;
    uint64_t n = 0;
    int nsm = 0;
    std::vector<uint64_t> hb2;
    QS3_TRY(enum_sorted_reps<ND>(B, K0, reps, stab, n, hb2, nsm));
    if (n >= (1ull << 20)) return set_err(QS3_ERR_OVERFLOW, "%llu orbits exceed the table's 20-bit index", (unsigned long long)n);
    if (ns * 4 + n * 4 * (uint64_t)B.S > max_bytes)
        return set_err(QS3_ERR_OOM, "representative table exceeds the limit");
    DevBuf orb, t2;
    QS3_TRY(orb.alloc(ns * 4));
    QS3_TRY(t2.alloc(n * 4 * (uint64_t)B.S));
    QS3_CUDA(cudaMemset(orb.p, 0xff, ns * 4));
    const size_t smem = (size_t)(B.nd + 3) * (B.N + 1) * 8 + (size_t)B.N * 4;
    QS3_CUDA(cudaFuncSetAttribute(k_orbit_fill<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM));
    const uint64_t tot = n * (uint64_t)B.ncell;
    int grid = (int)std::min<uint64_t>((tot + NTHREADS - 1) / NTHREADS, (uint64_t)nsm * 8);
    k_orbit_fill<ND><<<std::max(grid, 1), NTHREADS, smem>>>(B.lv, reps.as<uint64_t>(), n, orb.as<uint32_t>());
    QS3_LAUNCHED();
    const uint64_t tot2 = n * (uint64_t)B.S;
    int grid2 = (int)std::min<uint64_t>((tot2 + 255) / 256, (uint64_t)nsm * 8);
    k_orbit_rows<<<std::max(grid2, 1), 256>>>(B.d_secs.as<SecView>(), B.S, reps.as<uint64_t>(), n, t2.as<int32_t>());
    QS3_LAUNCHED();
    QS3_CUDA(cudaDeviceSynchronize());
    DevBuf phd;
    const uint64_t nph = (uint64_t)B.S * B.N;
    QS3_TRY(phd.alloc(nph * sizeof(int4)));
    k_phase_digits<<<(int)std::min<uint64_t>((nph + 255) / 256, 4096), 256>>>(B.d_ph64.as<double2>(), nph,
                                                                              phd.as<int4>());
    QS3_LAUNCHED();
    QS3_CUDA(cudaDeviceSynchronize());
    B.d_orb = std::move(orb);
    B.d_t2 = std::move(t2);
    B.d_oreps = std::move(reps);
    B.d_ostab = std::move(stab);
    B.d_phdig = std::move(phd);
    B.n_orb = n;
    B.lv.orb = B.d_orb.as<uint32_t>();
    B.lv.n_orb = (uint32_t)n;
    for (int s = 0; s < B.S; ++s) B.secs[s].t2 = B.d_t2.as<int32_t>() + (size_t)s * n;
    QS3_TRY(B.d_secs.upload(B.secs.data(), B.secs.size() * sizeof(SecView)));
    return QS3_OK;
}

int build_rep_table(Basis &B, size_t max_bytes) {
    if (!B.has_k || B.nd == 0 || B.total == 0) return set_err(QS3_ERR_STATE, "the table serves k-sector bases only");
    if (B.N > 4096) return set_err(QS3_ERR_OVERFLOW, "N > 4096");
    if (B.lv.orb) return QS3_OK;
    switch (B.nd) {
        case 1: return build_table_nd<1>(B, max_bytes);
        case 2: return build_table_nd<2>(B, max_bytes);
        case 3: return build_table_nd<3>(B, max_bytes);
        case 4: return build_table_nd<4>(B, max_bytes);
        case 5: return build_table_nd<5>(B, max_bytes);
        case 6: return build_table_nd<6>(B, max_bytes);
        case 7: return build_table_nd<7>(B, max_bytes);
        case 8: return build_table_nd<8>(B, max_bytes);
        default: return set_err(QS3_ERR_INVALID_ARG, "n_down %d", B.nd);
    }
}

void drop_rep_table(Basis &B) {
    B.lv.orb = nullptr;
    B.lv.n_orb = 0;
    for (auto &v : B.secs) v.t2 = nullptr;
    B.d_orb.release();
    B.d_t2.release();
    B.d_oreps.release();
    B.d_ostab.release();
    B.d_phdig.release();
    B.n_orb = 0;
    if (!B.secs.empty()) B.d_secs.upload(B.secs.data(), B.secs.size() * sizeof(SecView));
}

// per-sector phase tables ph[s N + r] = exp(-2 pi i sum_alpha K_alpha r_alpha / L_alpha):
// the phase e^{ik.t} of the translation t = -(r_x, r_y, r_z) that moves site r
// to the origin; the angle is reduced exactly in integers
// per sector s and cell translation u (u < G = Lx Ly Lz; rows of N entries,
// the entries past G repeat the table): e^{-2 pi i K.t_u / L} with the angle
// reduced exactly in integers
__global__ void k_phase_tables(int S, int N, int G, int Lx, int Ly, int Lz, const int *__restrict__ K,
                               double2 *__restrict__ ph64, float2 *__restrict__ ph32, float4 *__restrict__ phdf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * N) return;
    const int s = i / N, r = (i % N) % G;
    const long long x = r % Lx, y = (r / Lx) % Ly, z = r / (Lx * Ly);
    const long long num =
        ((long long)K[3 * s] * x * (G / Lx) + (long long)K[3 * s + 1] * y * (G / Ly) + (long long)K[3 * s + 2] * z * (G / Lz)) % G;
    double sn, cs;
    sincospi(-2.0 * (double)num / (double)G, &sn, &cs);
    ph64[i] = make_double2(cs, sn);
    ph32[i] = make_float2((float)cs, (float)sn);
    const float ch = __double2float_rn(cs), sh = __double2float_rn(sn);
    phdf[i] = make_float4(ch, __double2float_rn(cs - (double)ch), sh, __double2float_rn(sn - (double)sh));
}

// ---------------------------------------------------------------- host side

static bool binom_table(int N, int rows, std::vector<uint64_t> &t, uint64_t *cnd, int nd) {
    // t[m * (N+1) + c] = C(c, m), saturated at UINT64_MAX; returns false if C(N, nd) >= 2^63
    t.assign((size_t)rows * (N + 1), 0);
    for (int c = 0; c <= N; ++c) t[c] = 1;
    const uint64_t SAT = ~0ull;
    for (int m = 1; m < rows; ++m)
        for (int c = 1; c <= N; ++c) {
            uint64_t a = t[(size_t)(m - 1) * (N + 1) + c - 1], b = t[(size_t)m * (N + 1) + c - 1];
            uint64_t s = (a == SAT || b == SAT || a + b < a) ? SAT : a + b;
            t[(size_t)m * (N + 1) + c] = s;
        }
    *cnd = t[(size_t)nd * (N + 1) + N];
    return *cnd < (1ull << 63);
}

static int check_translation(const Basis &B) {
    // bonds as an unordered-pair multiset with summed couplings
    std::map<std::pair<int, int>, std::pair<double, double>> bonds;
    for (int b = 0; b < B.nb; ++b) {
        int i = std::min(B.bi[b], B.bj[b]), j = std::max(B.bi[b], B.bj[b]);
        auto &v = bonds[{i, j}];
        v.first += B.jxy[b];
        v.second += B.jz[b];
    }
    const int Lx = B.L[0], Ly = B.L[1], ns = B.nsub;
    // site r = spin r % ns of cell r / ns; the shift moves the cell by one along axis a
    auto shift = [&](int r, int a) {
        const int sb = r % ns, q = r / ns;
        int x = q % Lx, y = (q / Lx) % Ly, z = q / (Lx * Ly);
        if (a == 0) x = (x + 1) % Lx;
        if (a == 1) y = (y + 1) % Ly;
        if (a == 2) z = (z + 1) % B.L[2];
        return sb + ns * (x + Lx * (y + Ly * z));
    };
    for (int a = 0; a < 3; ++a) {
        if (B.L[a] == 1) continue;
        for (auto &kv : bonds) {
            int i = shift(kv.first.first, a), j = shift(kv.first.second, a);
            auto it = bonds.find({std::min(i, j), std::max(i, j)});
            if (it == bonds.end() || std::fabs(it->second.first - kv.second.first) > 1e-12 ||
                std::fabs(it->second.second - kv.second.second) > 1e-12)
                return set_err(QS3_ERR_SYMMETRY, "bond (%d,%d) is not invariant under the translation along axis %d",
                               kv.first.first, kv.first.second, a);
        }
    }
    // the field must be the same on every copy of a spin of the unit cell
    if (B.has_h)
        for (int i = 1; i < B.N; ++i)
            if (B.h[i] != B.h[i % ns]) return set_err(QS3_ERR_SYMMETRY, "site field is not translation invariant (site %d)", i);
    return QS3_OK;
}

static int basis_create(const qs3_lattice *lat, int nd, int nsec, const int32_t *K, Basis &B) {
    if (!lat) return set_err(QS3_ERR_INVALID_ARG, "lattice is NULL");
    const int N = lat->n_sites, nb = lat->n_bonds;
    if (N < 1 || N > QS3_MAX_SITES) return set_err(QS3_ERR_OVERFLOW, "n_sites %d outside [1, %d]", N, QS3_MAX_SITES);
    if (nd < 0 || nd > QS3_MAX_NDOWN || nd > N)
        return set_err(nd > QS3_MAX_NDOWN ? QS3_ERR_OVERFLOW : QS3_ERR_INVALID_ARG, "n_down %d", nd);
    if (nb < 0 || (nb > 0 && (!lat->bi || !lat->bj || !lat->jxy || !lat->jz)))
        return set_err(QS3_ERR_INVALID_ARG, "bond arrays");
    if (nsec < 1) return set_err(QS3_ERR_INVALID_ARG, "n_sectors %d", nsec);
    if (!K && nsec != 1) return set_err(QS3_ERR_INVALID_ARG, "a U(1)-only basis has exactly one sector");
    B.N = N;
    B.nd = nd;
    B.nb = nb;
    B.bi.assign(lat->bi, lat->bi + nb);
    B.bj.assign(lat->bj, lat->bj + nb);
    B.jxy.assign(lat->jxy, lat->jxy + nb);
    B.jz.assign(lat->jz, lat->jz + nb);
    for (int b = 0; b < nb; ++b) {
        if (B.bi[b] < 0 || B.bi[b] >= N || B.bj[b] < 0 || B.bj[b] >= N || B.bi[b] == B.bj[b])
            return set_err(QS3_ERR_INVALID_ARG, "bond %d joins (%d, %d)", b, B.bi[b], B.bj[b]);
        if (!std::isfinite(B.jxy[b]) || !std::isfinite(B.jz[b]))
            return set_err(QS3_ERR_INVALID_ARG, "bond %d has a non-finite coupling", b);
    }
    B.has_h = lat->h != nullptr;
    if (B.has_h) B.h.assign(lat->h, lat->h + N);
    for (int a = 0; a < 3; ++a) B.L[a] = lat->L[a];
    const bool haveL = B.L[0] > 0 || B.L[1] > 0 || B.L[2] > 0;
    B.nsub = lat->n_sub > 0 ? lat->n_sub : 1;
    if (haveL) {
        for (int a = 0; a < 3; ++a)
            if (B.L[a] < 1 || B.L[a] > (a == 2 ? 1023 : 2047))
                return set_err(QS3_ERR_INVALID_ARG, "L[%d] = %d outside the coordinate range", a, B.L[a]);
        if ((long long)B.nsub * B.L[0] * B.L[1] * B.L[2] != N)
            return set_err(QS3_ERR_INVALID_ARG, "n_sub*Lx*Ly*Lz = %lld != n_sites %d",
                           (long long)B.nsub * B.L[0] * B.L[1] * B.L[2], N);
    } else {
        if (B.nsub != 1) return set_err(QS3_ERR_INVALID_ARG, "n_sub %d without a translation group", B.nsub);
        if (N > 2047 && K) return set_err(QS3_ERR_INVALID_ARG, "translation group needed");
    }
    B.has_k = K != nullptr;
    B.S = nsec;
    if (B.has_k) {
        if (!haveL) return set_err(QS3_ERR_SYMMETRY, "momentum sectors need a translation group L");
        B.K.assign(K, K + 3 * nsec);
        for (int s = 0; s < nsec; ++s)
            for (int a = 0; a < 3; ++a)
                if (B.K[3 * s + a] < 0 || B.K[3 * s + a] >= B.L[a])
                    return set_err(QS3_ERR_SYMMETRY, "K[%d][%d] = %d outside [0, %d)", s, a, B.K[3 * s + a], B.L[a]);
        QS3_TRY(check_translation(B));
    } else {
        B.K.assign(3, 0);
    }
    if (!haveL) { B.L[0] = N; B.L[1] = 1; B.L[2] = 1; }
    B.ncell = B.L[0] * B.L[1] * B.L[2];
    if (lat->pos) B.pos.assign(lat->pos, lat->pos + 3 * (size_t)N);

    // binomial rows 0..nd+2
    std::vector<uint64_t> tb;
    uint64_t cnd = 0;
    if (!binom_table(N, nd + 3, tb, &cnd, nd))
        return set_err(QS3_ERR_OVERFLOW, "C(%d, %d) does not fit in 63 bits", N, nd);
    QS3_TRY(B.d_binom.upload(tb.data(), tb.size() * 8));

    // adjacency (CSR, both directions), diagonal constants
    std::vector<int> deg(N + 1, 0);
    for (int b = 0; b < nb; ++b) { deg[B.bi[b] + 1]++; deg[B.bj[b] + 1]++; }
    B.max_degree = 0;
    for (int i = 0; i < N; ++i) B.max_degree = std::max(B.max_degree, deg[i + 1]);
    for (int i = 0; i < N; ++i) deg[i + 1] += deg[i];
    std::vector<int> nbr(2 * (size_t)nb), fill(deg.begin(), deg.end() - 1);
    std::vector<double> ajxy(2 * (size_t)nb), ajz(2 * (size_t)nb), u(N, 0.0);
    std::vector<float> ajxyf(2 * (size_t)nb);
    double c0 = 0.0;
    for (int b = 0; b < nb; ++b) {
        int i = B.bi[b], j = B.bj[b];
        int p = fill[i]++, q = fill[j]++;
        nbr[p] = j; nbr[q] = i;
        ajxy[p] = ajxy[q] = 0.5 * B.jxy[b];            // hop amplitude J^xy / 2 of Eq. (1)
        ajz[p] = ajz[q] = B.jz[b];
        ajxyf[p] = ajxyf[q] = (float)(0.5 * B.jxy[b]);
        u[i] -= 0.5 * B.jz[b];
        u[j] -= 0.5 * B.jz[b];
        c0 += 0.25 * B.jz[b];
    }
    if (B.has_h)
        for (int i = 0; i < N; ++i) { u[i] += B.h[i]; c0 -= 0.5 * B.h[i]; }
    QS3_TRY(B.d_adj_ptr.upload(deg.data(), deg.size() * 4));
    QS3_TRY(B.d_adj_nbr.upload(nbr.data(), nbr.size() * 4));
    QS3_TRY(B.d_adj_jxy.upload(ajxy.data(), ajxy.size() * 8));
    QS3_TRY(B.d_adj_jz.upload(ajz.data(), ajz.size() * 8));
    QS3_TRY(B.d_adj_jxy_f.upload(ajxyf.data(), ajxyf.size() * 4));
    QS3_TRY(B.d_u.upload(u.data(), u.size() * 8));
    std::vector<float> uf(u.begin(), u.end()), ajzf(ajz.begin(), ajz.end());
    QS3_TRY(B.d_u_f.upload(uf.data(), uf.size() * 4));
    QS3_TRY(B.d_adj_jz_f.upload(ajzf.data(), ajzf.size() * 4));
    {
        // double-float remainders (v - fl32(v), rounded to fp32)
        auto rem = [](const std::vector<double> &v, const std::vector<float> &h) {
            std::vector<float> r(v.size());
            for (size_t i = 0; i < v.size(); ++i) r[i] = (float)(v[i] - (double)h[i]);
            return r;
        };
        const std::vector<float> a = rem(ajxy, ajxyf), bu = rem(u, uf), cz = rem(ajz, ajzf);
        QS3_TRY(B.d_adj_jxy_lo.upload(a.data(), a.size() * 4));
        QS3_TRY(B.d_u_lo.upload(bu.data(), bu.size() * 4));
        QS3_TRY(B.d_adj_jz_lo.upload(cz.data(), cz.size() * 4));
    }
    // fixed-width copy of the adjacency for the U(1) fp32 kernel
    const int padw = B.max_degree <= 4 ? 4 : (B.max_degree <= 6 ? 6 : 0);
    if (padw) {
        std::vector<int2> pk((size_t)N * padw);
        std::vector<float> pz((size_t)N * padw, 0.f);
        for (int i = 0; i < N; ++i)
            for (int b = 0; b < padw; ++b) {
                const int q = deg[i] + b;
                const bool real = q < deg[i + 1];
                float jf = real ? ajxyf[q] : 0.f;
                int bitsf;
                std::memcpy(&bitsf, &jf, 4);
                pk[(size_t)i * padw + b] = make_int2(real ? nbr[q] : i, bitsf);
                pz[(size_t)i * padw + b] = real ? ajzf[q] : 0.f;
            }
        QS3_TRY(B.d_adj_pad.upload(pk.data(), pk.size() * sizeof(int2)));
        QS3_TRY(B.d_adj_jz_pad.upload(pz.data(), pz.size() * 4));
    }
    std::vector<uint32_t> xyz(N);
    for (int r = 0; r < N; ++r) {
        // the coordinates of the site's cell
        const int q = r / B.nsub;
        int x = q % B.L[0], y = (q / B.L[0]) % B.L[1], z = q / (B.L[0] * B.L[1]);
        // coordinates are only used with a translation group (x, y < 2048, z < 1024)
        xyz[r] = haveL ? ((uint32_t)x | ((uint32_t)y << 11) | ((uint32_t)z << 22)) : 0u;
    }
    QS3_TRY(B.d_xyz.upload(xyz.data(), xyz.size() * 4));

    int bits = 1;
    while ((1 << bits) < N) ++bits;
    LatView &L = B.lv;
    L.N = N;
    L.nd = nd;
    L.np1 = N + 1;
    for (int a = 0; a < 3; ++a) L.L[a] = B.L[a];
    L.has_k = B.has_k;
    L.key_bits = (bits * nd <= 64) ? bits : 0;
    L.binom = B.d_binom.as<uint64_t>();
    L.adj_ptr = B.d_adj_ptr.as<int>();
    L.adj_nbr = B.d_adj_nbr.as<int>();
    L.adj_jxy = B.d_adj_jxy.as<double>();
    L.adj_jz = B.d_adj_jz.as<double>();
    L.adj_jxy_f = B.d_adj_jxy_f.as<float>();
    L.u = B.d_u.as<double>();
    L.c0 = c0;
    L.c0f = (float)c0;
    L.u_f = B.d_u_f.as<float>();
    L.adj_jz_f = B.d_adj_jz_f.as<float>();
    L.adj_jxy_lo = B.d_adj_jxy_lo.as<float>();
    L.u_lo = B.d_u_lo.as<float>();
    L.adj_jz_lo = B.d_adj_jz_lo.as<float>();
    L.c0lo = (float)(c0 - (double)(float)c0);
    L.xyz = B.d_xyz.as<uint32_t>();
    L.nsub = B.nsub;
    L.ncell = B.ncell;
    L.adj_pad = B.d_adj_pad.as<int2>();
    L.adj_jz_pad = B.d_adj_jz_pad.as<float>();
    L.pad_w = padw;
    L.jh_uniform = 0.0;
    if (nb > 0) {
        bool same = true;
        for (int b = 1; b < nb; ++b) same &= B.jxy[b] == B.jxy[0];
        if (same) L.jh_uniform = 0.5 * B.jxy[0];
    }

    // sectors
    B.dims.assign(nsec, 0);
    B.d_sigma.resize(nsec);
    B.d_stab.resize(nsec);
    B.d_pidx.resize(nsec);
    if (!B.has_k) {
        B.dims[0] = cnd;
    } else if (nd == 0) {
        for (int s = 0; s < nsec; ++s) {
            const bool k0 = B.K[3 * s] == 0 && B.K[3 * s + 1] == 0 && B.K[3 * s + 2] == 0;
            B.dims[s] = k0 ? 1 : 0;
            uint64_t zero = 0;
            uint8_t one = 1;
            uint32_t pi[2] = {0, k0 ? 1u : 0u};
            QS3_TRY(B.d_sigma[s].upload(&zero, 8));
            QS3_TRY(B.d_stab[s].upload(&one, 1));
            QS3_TRY(B.d_pidx[s].upload(pi, 8));
        }
    } else {
        for (int s = 0; s < nsec; ++s) QS3_TRY(build_sector_reps(B, s));
    }
    B.offs.assign(nsec + 1, 0);
    B.tile0.assign(nsec + 1, 0);
    B.chunk0.assign(nsec + 1, 0);
    for (int s = 0; s < nsec; ++s) {
        B.offs[s + 1] = B.offs[s] + B.dims[s];
        uint64_t nt = (B.dims[s] + TILE - 1) / TILE;
        if ((uint64_t)B.tile0[s] + nt > (1ull << 31) - 1) return set_err(QS3_ERR_OVERFLOW, "too many rows");
        B.tile0[s + 1] = B.tile0[s] + (int)nt;
        B.chunk0[s + 1] = B.chunk0[s] + (int)((B.dims[s] + BROWS - 1) / BROWS);
    }
    B.total = B.offs[nsec];
    B.ntiles = B.tile0[nsec];
    B.nchunks = B.chunk0[nsec];
    B.secs.resize(nsec);
    if (B.has_k) {
        QS3_TRY(B.d_ph64.alloc((size_t)nsec * N * sizeof(double2)));
        QS3_TRY(B.d_ph32.alloc((size_t)nsec * N * sizeof(float2)));
        QS3_TRY(B.d_phdf.alloc((size_t)nsec * N * sizeof(float4)));
        QS3_TRY(B.d_secs.upload(B.K.data(), B.K.size() * sizeof(int)));     // momenta for the table kernel
        const int tot = nsec * N;
        k_phase_tables<<<(tot + 255) / 256, 256>>>(nsec, N, B.ncell, B.L[0], B.L[1], B.L[2], B.d_secs.as<int>(),
                                                   B.d_ph64.as<double2>(), B.d_ph32.as<float2>(),
                                                   B.d_phdf.as<float4>());
        QS3_LAUNCHED();
        QS3_CUDA(cudaDeviceSynchronize());
    }
    for (int s = 0; s < nsec; ++s) {
        SecView &v = B.secs[s];
        v.sigma = B.has_k ? B.d_sigma[s].as<uint64_t>() : nullptr;
        v.stab = B.has_k ? B.d_stab[s].as<uint8_t>() : nullptr;
        v.pidx = B.has_k ? B.d_pidx[s].as<uint32_t>() : nullptr;
        v.dim = B.dims[s];
        v.off = B.offs[s];
        for (int a = 0; a < 3; ++a) v.K[a] = B.K[3 * s + a];
        v.tile0 = B.tile0[s];
        v.ph64 = B.has_k ? B.d_ph64.as<double2>() + (size_t)s * N : nullptr;
        v.ph32 = B.has_k ? B.d_ph32.as<float2>() + (size_t)s * N : nullptr;
        v.phdf = B.has_k ? B.d_phdf.as<float4>() + (size_t)s * N : nullptr;
    }
    QS3_TRY(B.d_secs.upload(B.secs.data(), B.secs.size() * sizeof(SecView)));
    QS3_TRY(B.d_tile0.upload(B.tile0.data(), B.tile0.size() * 4));
    QS3_TRY(B.d_chunk0.upload(B.chunk0.data(), B.chunk0.size() * 4));
    B.smem_bytes = row_kernel_smem(B, 0);
    if (B.smem_bytes > 200 * 1024)
        return set_err(QS3_ERR_OVERFLOW, "lattice tables need %zu bytes of shared memory", B.smem_bytes);
    B.narrow_ranks = !B.has_k && nd >= 1 && B.total > 0 && B.total < (1ull << 32);
    // the representative table when it is small (a bounded fraction of the
    // device memory); otherwise H Phi runs the representative search
    if (B.has_k && nd > 0 && B.total > 0 && N <= 4096) {
        size_t fr = 0, tt = 0;
        QS3_CUDA(cudaMemGetInfo(&fr, &tt));
        const size_t lim = std::min<size_t>(REP_TABLE_AUTO_BYTES, fr / 8);
        if (build_rep_table(B, lim) != QS3_OK) {
            drop_rep_table(B);
            clear_err();
        }
    }
    return QS3_OK;
}

}  // namespace qs3

using namespace qs3;

extern "C" {

int qs3_basis_create(const qs3_lattice *lat, int32_t n_down, int32_t n_sectors, const int32_t *K, qs3_basis_t *out) {
    clear_err();
    if (!out) return set_err(QS3_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    qs3_basis_s *h = new (std::nothrow) qs3_basis_s();
    if (!h) return set_err(QS3_ERR_OOM, "host allocation");
    int st = basis_create(lat, n_down, n_sectors, K, h->B);
    if (st != QS3_OK) {
        delete h;
        return st;
    }
    *out = h;
    return QS3_OK;
}

int qs3_basis_destroy(qs3_basis_t b) {
    clear_err();
    delete b;
    return QS3_OK;
}

int qs3_basis_info(qs3_basis_t b, int32_t *n_sectors, uint64_t *total_dim) {
    clear_err();
    if (!b) return set_err(QS3_ERR_INVALID_ARG, "basis is NULL");
    if (n_sectors) *n_sectors = b->B.S;
    if (total_dim) *total_dim = b->B.total;
    return QS3_OK;
}

int qs3_basis_dims(qs3_basis_t b, uint64_t *dims) {
    clear_err();
    if (!b || !dims) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    for (int s = 0; s < b->B.S; ++s) dims[s] = b->B.dims[s];
    return QS3_OK;
}

int qs3_basis_ranks(qs3_basis_t b, int32_t s, uint64_t *ranks, uint8_t *stab) {
    clear_err();
    if (!b || !ranks) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    Basis &B = b->B;
    if (s < 0 || s >= B.S) return set_err(QS3_ERR_INVALID_ARG, "sector %d", s);
    if (!B.has_k) return set_err(QS3_ERR_INVALID_ARG, "a U(1)-only sector has ranks 0..dim-1");
    if (B.dims[s]) {
        QS3_CUDA(cudaMemcpy(ranks, B.d_sigma[s].p, B.dims[s] * 8, cudaMemcpyDeviceToHost));
        if (stab) QS3_CUDA(cudaMemcpy(stab, B.d_stab[s].p, B.dims[s], cudaMemcpyDeviceToHost));
    }
    return QS3_OK;
}

int qs3_basis_nnz(qs3_basis_t b, uint64_t *nnz) {
    clear_err();
    if (!b || !nnz) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    QS3_TRY(count_nnz(b->B, nnz));
    return QS3_OK;
}

int qs3_basis_rep_table(qs3_basis_t b, int32_t mode, int32_t *active) {
    clear_err();
    if (!b) return set_err(QS3_ERR_INVALID_ARG, "basis is NULL");
    if (mode < -1 || mode > 1) return set_err(QS3_ERR_INVALID_ARG, "mode %d", mode);
    int st = QS3_OK;
    if (mode == 0) {
        drop_rep_table(b->B);
    } else if (mode == 1) {
        size_t fr = 0, tt = 0;
        QS3_CUDA(cudaMemGetInfo(&fr, &tt));
        st = build_rep_table(b->B, fr - fr / 16);
        if (st != QS3_OK) {
            std::string msg = last_err();
            drop_rep_table(b->B);
            set_err(st, "%s", msg.c_str());
        }
    }
    if (active) *active = b->B.lv.orb ? 1 : 0;
    return st;
}

int qs3_basis_tuning(qs3_basis_t b, int32_t set, int32_t *hphi_blocks_per_sm, int32_t *dot_vectors,
                     int32_t *dot_vectors64) {
    clear_err();
    if (!b) return set_err(QS3_ERR_INVALID_ARG, "basis is NULL");
    Basis &B = b->B;
    auto nv_ok = [](const int32_t *v) { return !v || *v == 0 || *v == 1 || *v == 2 || *v == 4; };
    auto nv64_ok = [&](const int32_t *v) { return nv_ok(v) || *v == 8; };
    if (set) {
        if (hphi_blocks_per_sm)
            for (int i = 0; i < 5; ++i)
                if (hphi_blocks_per_sm[i] < 0) return set_err(QS3_ERR_INVALID_ARG, "blocks per SM %d", hphi_blocks_per_sm[i]);
        if (!nv_ok(dot_vectors)) return set_err(QS3_ERR_INVALID_ARG, "dot vectors per pass %d", *dot_vectors);
        if (!nv64_ok(dot_vectors64)) return set_err(QS3_ERR_INVALID_ARG, "dot vectors per pass %d", *dot_vectors64);
        if (hphi_blocks_per_sm)
            for (int i = 0; i < 5; ++i) B.tune_hphi[i] = hphi_blocks_per_sm[i];
        if (dot_vectors) B.tune_nv = *dot_vectors;
        if (dot_vectors64) B.tune_nv64 = *dot_vectors64;
    } else {
        if (hphi_blocks_per_sm)
            for (int i = 0; i < 5; ++i) hphi_blocks_per_sm[i] = B.tune_hphi[i];
        if (dot_vectors) *dot_vectors = B.tune_nv;
        if (dot_vectors64) *dot_vectors64 = B.tune_nv64;
    }
    return QS3_OK;
}

int64_t qs3_inject_alloc_failure(int64_t after) {
    return (int64_t)qs3::g_alloc_budget.exchange(after < 0 ? -1 : (long long)after);
}

int32_t qs3_inject_wait_timeout(int32_t n) { return qs3::g_wait_starve.exchange(n > 0 ? n : 0); }

const char *qs3_last_error(void) { return qs3::last_err(); }

const char *qs3_strerror(int status) {
    switch (status) {
        case QS3_OK: return "ok";
        case QS3_ERR_INVALID_ARG: return "invalid argument";
        case QS3_ERR_OVERFLOW: return "size overflow";
        case QS3_ERR_SYMMETRY: return "symmetry violated";
        case QS3_ERR_OOM: return "out of device memory";
        case QS3_ERR_CUDA: return "CUDA error";
        case QS3_ERR_NOT_CONVERGED: return "not converged";
        case QS3_ERR_TIMEOUT: return "device wait timed out";
        case QS3_ERR_STATE: return "invalid state";
        default: return "unknown status";
    }
}

const char *qs3_version(void) { return "qs3-gb300 0.1 (sm_103a)"; }

uint64_t qs3_kernel_launches(void) { return qs3::g_launches.load(); }

}  // extern "C"
