/*
 * qs3.h -- C ABI of libqs3.so, a GB300 (sm_103a) implementation of the hot
 * path of QS^3 (Ueda, Yunoki, Shimokawa, "Quantum spin solver near
 * saturation"): the matrix-free product H Phi of the spin-1/2 XXZ model in the
 * basis fixed by the number N_down of down spins and the wave number k, the
 * Lanczos / thick-restart Lanczos iteration that drives it, two-point
 * functions, S(q) and the continued-fraction S(q, omega).
 *
 * Conventions (all calls):
 *  - Sites are 0-based.  With a translation group (L[0], L[1], L[2]) the
 *    site index is r = x + Lx (y + Ly z) and T^t moves site coordinates by
 *    +t modulo L.
 *  - A U(1) basis state is the ascending list c_1 < ... < c_Nd of its
 *    down-spin sites; its rank is rank0 = sum_m C(c_m, m) (m = 1..Nd), the
 *    paper's index a of Eq. (a_of_n) minus one.  No bit strings are used.
 *  - A k-sector is the list sigma of representatives (minimum rank over the
 *    translation orbit, Sec. "Representative states ...") that are
 *    compatible with K, sorted by rank, with |Stab| of each; the
 *    normalisation factor of Eq. (akstate) is N_{a,k} = N |Stab(a)|.
 *    The momentum is k.a_alpha = 2 pi K_alpha / L_alpha.
 *  - A basis handle holds one or more sectors of one lattice and one N_down
 *    (several K at once, or one U(1)-only sector).  A vector on a basis is
 *    the concatenation of its sectors' vectors, sector s starting at the
 *    offset given by qs3_basis_dims (prefix sums).
 *  - Vectors are caller-owned DEVICE pointers (e.g. torch tensors) of the
 *    stated qs3_dtype; complex types are interleaved (re, im).  The library
 *    never frees them.  Host outputs go to caller arrays of the stated sizes.
 *  - stream arguments are cudaStream_t passed as void* (NULL = default
 *    stream); calls that return host data synchronise that stream.
 *  - Every call returns QS3_OK (0) or a negative status; no exception crosses
 *    the ABI and the library never exits the process.  qs3_last_error()
 *    returns a thread-local text describing the last failure.
 */
#ifndef QS3_H
#define QS3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QS3_MAX_NDOWN 8        /* largest N_down handled by the kernels        */
#define QS3_MAX_SITES 4096     /* largest N handled by the kernels             */

enum {
    QS3_OK = 0,
    QS3_ERR_INVALID_ARG = -1,   /* bad pointer, size, bond or option            */
    QS3_ERR_OVERFLOW = -2,      /* C(N, N_down) >= 2^63, N_down or N too large  */
    QS3_ERR_SYMMETRY = -3,      /* bonds/field not translation invariant, K out of range */
    QS3_ERR_OOM = -4,           /* device allocation failed                     */
    QS3_ERR_CUDA = -5,          /* a CUDA call failed                           */
    QS3_ERR_NOT_CONVERGED = -6, /* iteration limit reached before convergence   */
    QS3_ERR_TIMEOUT = -7,       /* a bounded device wait gave up                */
    QS3_ERR_STATE = -8          /* handle in the wrong state / dtype mismatch    */
};

/* Vector types of qs3_hphi.  QS3_C128DF: phi holds each complex element in
 * double-float form, four floats (re.hi, re.lo, im.hi, im.lo) with re =
 * re.hi + re.lo (qs3_split_df makes it from complex128); psi is complex128;
 * the product runs in double-float arithmetic (error-free fp32 products and
 * two-sums, about 48 significant bits), k-sector bases only.
 * QS3_C128X: phi and psi complex128; the product of the binary64 engine on
 * the integer units (k-sector bases with the representative table and one
 * hop amplitude on every bond): each hop's phase x phi formed exactly on
 * fixed-point images (phi rounded to 2^-53 of the largest magnitude among
 * its 128-row warp group, the phases to 2^-53), summed per row in a 64-bit
 * integer on the grid of the row's largest term (each term rounded once to
 * it) and rounded to binary64 once; terms whose target stabiliser differs
 * from the row's, and the diagonal, in binary64. */
typedef enum { QS3_F32 = 0, QS3_F64 = 1, QS3_C64 = 2, QS3_C128 = 3, QS3_C128DF = 4, QS3_C128X = 5 } qs3_dtype;

/* S^alpha_q operators, numbered as the paper's input parameter spsmsz. */
typedef enum { QS3_OP_SPLUS = 1, QS3_OP_SMINUS = 2, QS3_OP_SZ = 3 } qs3_sq_op;

/* Lattice and couplings of Eq. (1): H = sum_b [Jxy_b (s^x s^x + s^y s^y) +
 * Jz_b s^z s^z] - sum_i h_i s^z_i.  Bond b joins sites bi[b] != bj[b]; a
 * repeated pair adds its couplings.  h may be NULL (no field).  L = {0,0,0}
 * means no translation group (U(1) only).  Otherwise L is the translation
 * group of the unit cells and n_sub the spins per cell (0 or 1: a Bravais
 * lattice, one spin per cell; more: the multi-spin cells the paper's Summary
 * names, e.g. honeycomb or kagome): site r is spin r % n_sub of the cell
 * r / n_sub, cells numbered x + Lx (y + Ly z), T^t moves every cell by +t
 * and keeps each spin's place in its cell, and n_sub*Lx*Ly*Lz must equal
 * n_sites.  pos (3*n_sites doubles, in lattice units) gives the site
 * positions used by e^{-i q.r}; NULL means the cell coordinates (x, y, z).
 * The S^alpha_q operators, S(q, omega) and the translation-symmetrised
 * correlations of k-sectors take one spin per cell, and S(q) of a lattice
 * with several needs pos (INVALID_ARG otherwise).
 * All pointers are host pointers and are copied; the caller keeps them. */
typedef struct {
    int32_t n_sites, n_bonds;
    const int32_t *bi, *bj;
    const double *jxy, *jz;
    const double *h;
    int32_t L[3];
    const double *pos;
    int32_t n_sub;
    int32_t reserved;
} qs3_lattice;

typedef struct qs3_basis_s *qs3_basis_t;

/* Build a basis for N_down down spins (Sec. "Representation of states with the
 * U(1) symmetry"; Alg. 5-6 for k-sectors).  K = NULL: one U(1)-only sector of
 * dimension C(N, N_down) (n_sectors must be 1).  Otherwise K holds 3 ints per
 * sector (K_alpha in [0, L_alpha)); the representative lists are enumerated,
 * filtered and sorted on the device.  Errors: INVALID_ARG, OVERFLOW,
 * SYMMETRY (bonds or h not invariant under the translations, K out of range),
 * OOM, CUDA.  The handle owns its device memory until qs3_basis_destroy. */
int qs3_basis_create(const qs3_lattice *lat, int32_t n_down, int32_t n_sectors, const int32_t *K,
                     qs3_basis_t *out);
int qs3_basis_destroy(qs3_basis_t b);

/* n_sectors and the total dimension (sum over sectors). */
int qs3_basis_info(qs3_basis_t b, int32_t *n_sectors, uint64_t *total_dim);
/* dims[s] for s < n_sectors (host array). */
int qs3_basis_dims(qs3_basis_t b, uint64_t *dims);
/* Sector s: rank0 of each representative (sorted), copied to a host array of
 * dims[s] entries; stab (may be NULL) receives |Stab| per representative.
 * INVALID_ARG for a U(1)-only sector (its ranks are 0..dim-1). */
int qs3_basis_ranks(qs3_basis_t b, int32_t s, uint64_t *ranks, uint8_t *stab);
/* Number of structural non-zeros of H on the basis: the diagonal plus every
 * off-diagonal term of Alg. 9 that lands on a member of the sector.  Counted
 * once on the device and cached. */
int qs3_basis_nnz(qs3_basis_t b, uint64_t *nnz);
/* Representative table of a k-sector basis.  The representative search of
 * Alg. 7 (with the sigma lookup of Alg. 9) is a fixed function of the state;
 * for lattices whose C(N, N_down) states fit a 4-byte table it can be
 * tabulated once: for every state, by rank0, its orbit and the translation
 * to the representative, plus per sector the row of every orbit.  H Phi then
 * uses two table loads per hop target instead of the search; the results are
 * identical.  The table is built at qs3_basis_create when it needs at most
 * 1 GiB and an eighth of the free device memory.
 *   mode = 1: build it (any size that fits); OVERFLOW when C(N, N_down) >= 2^32
 *             or there are 2^20 orbits or more, OOM when it does not fit,
 *             STATE on a U(1)-only basis or N_down = 0;
 *   mode = 0: release it (H Phi runs the search);
 *   mode = -1: query only.
 * *active (may be NULL) receives 1 if the table is in use afterwards.  The
 * table occupies C(N, N_down) * 4 + n_sectors * n_orbits * 4 bytes of device
 * memory, library-owned, released with the basis. */
int qs3_basis_rep_table(qs3_basis_t b, int32_t mode, int32_t *active);
/* Autotuned launch choices of a basis (no counterpart in the paper).  On the
 * first direct (not stream-captured) use, the library times:
 *   - H Phi with 1..4 fewer resident 256-row blocks per SM than the occupancy
 *     limit (the persistent grid, i.e. rows in flight per SM), per vector
 *     dtype, and keeps the fastest;
 *   - the dot products of the Gram-Schmidt pass with 1, 2 or 4 basis vectors
 *     per pass (loads in flight together): dot_vectors for the double-float
 *     engine and the fp32 phase, dot_vectors64 for the binary64 engine, which
 *     also has 8: the stored vectors' digits copied by bulk asynchronous
 *     copies (TMA) into rings in shared memory, for the dot pass (k_dotb)
 *     and for the Gram-Schmidt update (k_updb).
 * set = 0: write the current choices (0 = not tuned yet) to
 *          hphi_blocks_per_sm[5] (indexed by qs3_dtype), *dot_vectors and
 *          *dot_vectors64;
 * set = 1: impose them (0 = tune again at the next use; blocks per SM above
 *          the occupancy limit are clamped; vectors per pass in {0, 1, 2, 4},
 *          and 8 for dot_vectors64; INVALID_ARG otherwise).
 * Any pointer may be NULL.  Results do not depend on the choices. */
int qs3_basis_tuning(qs3_basis_t b, int32_t set, int32_t *hphi_blocks_per_sm, int32_t *dot_vectors,
                     int32_t *dot_vectors64);
/* Stored terms of a k-sector basis (an opt-in variant of Alg. 9, which the
 * paper recomputes matrix-free on every product).  mode = 1 enumerates every
 * off-diagonal term once -- its target row, the translation to the target's
 * representative, the target's |Stab| and the bond -- in the order H Phi
 * visits them, plus each row's diagonal; later qs3_hphi calls (and the
 * solvers) then gather from this list instead of searching representatives.
 * C128 results are identical bit for bit to the matrix-free product; C64
 * rounds the stored fp64 diagonal once.  Memory: 8 bytes per term + 16 bytes
 * per row, library-owned, at most half the free device memory (OOM beyond).
 * mode = 0 releases it, mode = -1 queries.  *bytes (may be NULL) receives the
 * device bytes held.  Errors: STATE (U(1)-only basis or N_down = 0),
 * OVERFLOW (N > 4096 or 32768 bonds or more), OOM. */
int qs3_basis_store_terms(qs3_basis_t b, int32_t mode, uint64_t *bytes);

/* psi = H phi (Alg. 9, pull form, one row per thread, no atomics).
 * dtype: F32/F64 on a U(1)-only basis (real H); C64/C128 on any basis;
 * C128DF (phi double-float, psi complex128) on a basis with momentum
 * sectors, within a few 2^-48 relative of the exact product per term.
 * phi and psi are device vectors of the basis' total dimension and must not
 * alias.  F32/C64 use fp32 matrix elements and fp32 row accumulation.
 * C128X allocates device scratch of twice the vector size per call.
 * Errors: STATE (real dtype on a k-sector basis, C128DF on a U(1)-only one,
 * C128X without the representative table or with bond-dependent J^xy). */
int qs3_hphi(qs3_basis_t b, qs3_dtype dtype, const void *phi, void *psi, void *stream);

/* Dot products of the Gram-Schmidt pass of Alg. 10 (the reorthogonalisation
 * of a new Lanczos vector against the stored ones), per sector:
 * out[2 (s m + j)], out[2 (s m + j) + 1] = re, im of conj(V_j) . w summed
 * over the rows of sector s, V_j = V + j ldv elements, j < m.  dtype F64
 * (real vectors, im = 0) or C128 (interleaved re, im); V and w are device
 * binary64 vectors of the basis' total dimension, out is host memory of
 * 2 S m doubles, written when the call returns (synchronous on stream).
 * mode 0 (the dots of fp64 solves): every operand is rounded once onto a
 * fixed-point grid set by the largest exponent among the 128 rows of its
 * warp (rows r with the same r mod 2048 div 32 within a chunk of 2048),
 * at most 2^-53 of that largest magnitude, and split into two balanced
 * digits (weights 2^26 and 1); the top x top and the cross digit products
 * are summed exactly in 64-bit integers, the low x low ones dropped, each
 * thread's cross sum rounded to the nearest multiple of 2^26; the warps'
 * sums are aligned to the coarsest grid of the sector (rounded to nearest)
 * and added exactly in 128-bit integers, and each sector's dot is rounded
 * to binary64 once.  The pass is the one the basis' dot_vectors64 choice
 * selects (qs3_basis_tuning; 2 when untuned): the results are the same bits
 * for every choice.
 * mode 1 (strict64 solves): binary64 FMA chains per thread, summed in a
 * fixed order.  Device scratch of m x the vector size is allocated per call.
 * Errors: INVALID_ARG (NULL, m < 0, ldv < total dimension for m > 1, dtype,
 * mode), OOM, TIMEOUT (a bounded wait of the copy ring ran out; the context
 * stays usable). */
int qs3_gs_dots(qs3_basis_t b, qs3_dtype dtype, int32_t m, const void *V, uint64_t ldv, const void *w,
                double *out, int32_t mode, void *stream);

/* x_df[r] = double-float split of the complex128 x[r], r < n: re.hi =
 * fl32(re), re.lo = fl32(re - re.hi), the same for im (device pointers, the
 * layout QS3_C128DF reads). */
int qs3_split_df(const void *x, void *x_df, uint64_t n, void *stream);

/* Options of the eigensolvers (input_lancz / input_TRLan of the paper). */
typedef struct {
    int32_t n_eig;        /* NOE: eigenpairs wanted per sector (TRL), 1 for Lanczos */
    int32_t n_keep;       /* N_K of Alg. 10 */
    int32_t n_max;        /* N_M of Alg. 10; for qs3_lanczos the largest Krylov size */
    int32_t max_iter;     /* I_M (restarts) for TRL; unused by qs3_lanczos */
    int32_t min_iter;     /* minitr: Lanczos steps before the first check */
    int32_t check_every;  /* itrint: steps between convergence checks */
    double eps;           /* lnc_ene_conv: relative Ritz-value change for convergence */
    int32_t precision;    /* QS3_F64: IEEE binary64 (complex double on k-sector bases): Lanczos vectors
                             stored as binary64, updates on binary64 FMAs, dot products and (k-sector
                             bases with the representative table and one hop amplitude) the H Phi
                             products summed exactly on 53-bit fixed-point images of the operands
                             (see qs3_gs_dots, QS3_C128X and strict64);
                             QS3_F32: fp32 vectors and H Phi with fp32 row sums, fp64 alpha/beta and
                             dot products (double-float sums of exact fp32 products), then a QS3_F64
                             refinement from the fp32 Ritz vectors;
                             QS3_C128DF: the double-float engine, a faster variant below binary64: the
                             Krylov basis stored as pairs of fp32 (about 48 significant bits, fp32
                             exponent range) and, on k-sector bases, H Phi, three-term part and
                             Gram-Schmidt in double-float arithmetic on the fp32 units */
    int32_t use_graphs;   /* fp64 solves: replay each Lanczos step (after the first) as a CUDA graph
                             captured once per vector-ring phase; fp32 vectors ignore it */
    uint64_t seed;        /* start vector: seeded Gaussian (SplitMix64 + Box-Muller) */
    double refine_tol;    /* fp32 mode: refine until |dE| <= refine_tol |E| (e.g. 1e-9) */
    double res_tol;       /* qs3_lanczos also needs the Ritz residual beta_m |c_m| <= res_tol max(|E|, 1); 0 = off */
    int32_t hphi_ieee;    /* precision QS3_C128DF on k-sector bases: 0 applies H to the double-float copy
                             of each Lanczos vector in double-float arithmetic; 1 uses the IEEE
                             complex128 H Phi.  Residuals are always IEEE binary64. */
    int32_t strict64;     /* QS3_F64 engine: 0 computes the dot products (qs3_gs_dots mode 0) and the
                             H Phi products (QS3_C128X) exactly on fixed-point images and lets the
                             Gram-Schmidt update whose m
                             coefficients are below 2^-40 |w| in sum (times 256 / m for m > 256)
                             form its correction in fp32 from the images' top digits (error below
                             2^-55.5 |w|, less than binary64 rounding of w); 1 keeps H Phi, the
                             dot products and every update on binary64 FMAs */
} qs3_solve_opts;

typedef struct {
    int32_t iterations;   /* H Phi applications (Lanczos steps), all phases */
    int32_t restarts;     /* thick restarts performed */
    int32_t converged;    /* sectors that met the criterion */
    int32_t refine_iterations; /* fp64 Lanczos steps spent in refinement */
    double max_residual;  /* max over sectors/eigenpairs of ||H v - E v|| (fp64, unit v) */
    double seconds;       /* wall time of the call */
    uint64_t hphi_nnz;    /* structural non-zeros applied by the H Phi launches (active sectors only) */
    double hphi_seconds;  /* device time of the H Phi launches outside CUDA graphs (CUDA events on the call's stream) */
    int32_t hphi_calls;   /* H Phi launches */
    int32_t hphi_graph_calls; /* of which replayed inside CUDA graphs (not in hphi_seconds) */
    double gs_dot_seconds;    /* device time of the Gram-Schmidt dot-product launches outside CUDA graphs */
    uint64_t gs_dot_bytes;    /* their algorithmic bytes: stored basis vectors and w read, active sectors */
    int32_t gs_dot_calls;     /* those launches */
    int32_t reserved;
    uint64_t gs_dot_fma;      /* binary64 engine: the real multiply-adds those launches stand for (4 per
                                 complex element and stored vector, 1 per real one; binary64 FMAs
                                 under strict64, integer digit products otherwise); 0 for the other
                                 engines */
} qs3_solve_info;

/* Conventional Lanczos with full reorthogonalisation (Alg. 10 lines 2-12)
 * to the lowest eigenpair of every sector, batched over the sectors.  The
 * QS3_F64 engine takes the recurrence as printed (alpha_x = Re psi_x^H v,
 * v - alpha_x psi_x - beta_{x-1} psi_{x-1}) and then one classical
 * Gram-Schmidt pass against every stored vector.
 * evals: host, n_sectors doubles.  evecs: device fp64 vector (F64 for a
 * U(1)-only basis, C128 otherwise) of the total dimension, or NULL.
 * Returns NOT_CONVERGED when n_max steps did not meet eps (results are the
 * last Ritz values), TIMEOUT when a bounded wait of a copy ring ran out (see
 * qs3_inject_wait_timeout; the context stays usable). */
int qs3_lanczos(qs3_basis_t b, const qs3_solve_opts *o, double *evals, void *evecs, qs3_solve_info *info,
                void *stream);

/* Thick-restart Lanczos (Alg. 10) for the n_eig lowest eigenpairs of every
 * sector, batched.  evals: host, n_sectors * n_eig (sector-major).  evecs:
 * device, n_eig fp64 vectors of the total dimension one after another, or
 * NULL.  The first step after a restart removes the arrowhead couplings by
 * a full first pass; errors as qs3_lanczos. */
int qs3_trlanczos(qs3_basis_t b, const qs3_solve_opts *o, double *evals, void *evecs, qs3_solve_info *info,
                  void *stream);

/* Lowest eigenpair of every sector of n independent bases (different
 * lattices, N_down and momenta), solved concurrently with the options of
 * qs3_lanczos: host workers each drive their own CUDA stream, take the
 * instances largest first, and start one only when its Lanczos storage fits
 * the device's free memory next to those in flight.  evals: host, the
 * instances' sectors one after another (sum of n_sectors doubles).  evecs:
 * NULL or n device pointers (each NULL or an fp64 vector of that basis'
 * total dimension).  infos: NULL or n entries.  max_concurrent <= 0 means 16.
 * Returns the first failure (text in qs3_last_error), NOT_CONVERGED if any
 * instance did not converge. */
int qs3_batch_solve(int32_t n, const qs3_basis_t *bases, const qs3_solve_opts *o, double *evals,
                    void *const *evecs, qs3_solve_info *infos, int32_t max_concurrent);

/* Two-point functions of a state gs (device, fp64: F64 on a U(1)-only basis,
 * C128 otherwise) living in sector s of b (Sec. "Calculating expectation
 * values").  For k-sectors the translation-symmetrised operators are used, so
 * results depend on bj - bi only.  For each of n_pairs pairs (i, j) (host
 * 2*n_pairs ints): szsz[p] = <s^z_i s^z_j>, spsm[2p..2p+1] = <s^+_i s^-_j>
 * (re, im).  sz_local (n_sites or NULL) = <s^z_i>.  For each of n_q wave
 * vectors (host, 3 doubles each: q.a_alpha in radians): sq_zz[n] =
 * (1/N) sum_{r,r'} e^{iq.(r-r')} <s^z_r s^z_r'> and sq_pm[n] = the same for
 * <s^+_r s^-_r'>.  Any output may be NULL. */
int qs3_correlations(qs3_basis_t b, int32_t s, const void *gs, int32_t n_pairs, const int32_t *pairs,
                     double *szsz, double *spsm, double *sz_local, int32_t n_q, const double *q,
                     double *sq_zz, double *sq_pm, void *stream);

/* S^-_q applied to a state (Alg. 11, pull form): src sector s_src of basis
 * src (N_down, K) -> sector s_dst of basis dst (N_down + 1, K + Q), with
 * Q[3] the integer momentum of q (q.a_alpha = 2 pi Q_alpha / L_alpha).
 * phi, psi: device C128 vectors of the respective sector dimensions.  For a
 * U(1)-only pair of bases Q still fixes q through L; a lattice given with
 * L = {0,0,0} is numbered as a chain (L = {N,1,1}), so Q[0] then gives
 * q = 2 pi Q[0] / N along the site index, and Q = {0,0,0} gives q = 0. */
int qs3_smq(qs3_basis_t src, int32_t s_src, const void *phi, qs3_basis_t dst, int32_t s_dst, const int32_t *Q,
            void *psi, void *stream);

/* qs3_smq for callers that must not allocate device memory during the call:
 * code that hands all device memory out of its own pool, or that runs where
 * an allocation would synchronise the device.  The paper has no counterpart;
 * the result equals qs3_smq's.  The call allocates nothing: its one scratch
 * array, the site phases e^{-i q.R}, is a fixed 32 KB device array
 * inside the library that every GPU using the library keeps until the
 * process exits.  Limits: n_sites <= 2048 (QS3_ERR_INVALID_ARG beyond) and
 * lattices without a pos array (positions are the coordinates).  The first
 * call on a device looks that array up (cudaGetSymbolAddress), so make it
 * before any stream capture.  All calls share the array: two calls that
 * overlap on the GPU (different streams, or graphs replayed concurrently)
 * race; calls ordered on one stream do not.  The call is asynchronous on
 * stream. */
int qs3_smq_noalloc(qs3_basis_t src, int32_t s_src, const void *phi, qs3_basis_t dst, int32_t s_dst,
                    const int32_t *Q, void *psi, void *stream);

/* Dynamical structure factor S^-(q, omega) by the continued fraction of
 * Eq. (cfe) from n_iter Lanczos steps (fully reorthogonalised) started from
 * S^-_q |gs>, for n_q momenta at once (batched).  gs: device C128 state of
 * sector s_src of src with energy e0 (field-free).  dst must hold, in order,
 * the n_q sectors (N_down + 1, K + Q_n).  Q: host, 3*n_q ints.  The field
 * h_field enters as the Zeeman shift of the resolvent (poles at
 * E_n - e0 + h_field).  Outputs (host, may be NULL): s_qw[n*n_omega + w],
 * alpha[n*n_iter + x], beta[n*n_iter + x] (beta[n*n_iter] is |S^-_q gs|,
 * beta[x] for x >= 1 the Lanczos couplings), norm2[n] = |S^-_q gs|^2. */
int qs3_dsf(qs3_basis_t src, int32_t s_src, const void *gs, double e0, qs3_basis_t dst, int32_t n_q,
            const int32_t *Q, int32_t n_iter, double eta, double h_field, int32_t n_omega, const double *omega,
            double *s_qw, double *alpha, double *beta, double *norm2, void *stream);

/* S^alpha_q phi for alpha = op (qs3_sq_op), with S^alpha_q = N^{-1/2}
 * sum_j e^{-i q.R_j} S^alpha_j (Eq. sq_phi; the paper applies S^+_q and S^z_q
 * "in the same manner" as Alg. 11).  src sector s_src (N_down, K) -> dst
 * sector s_dst (N_down - 1 for S^+, N_down + 1 for S^-, N_down for S^z;
 * momentum K + Q).  Pull forms: S^z_q keeps the representative, a row b
 * taking N^{-1/2} (sum_j e^{-iq.R_j}/2 - sum_{j in b} e^{-iq.R_j}) phi_b (0 if
 * b is not in the source sector); S^+_q sums a row over its up sites s with
 * the representative of b + {s}, its translation phase and norm ratio.
 * op = QS3_OP_SMINUS is qs3_smq.  phi, psi: device C128 vectors of the
 * sector dimensions (NULL allowed for an empty sector); the call
 * synchronises stream.  Errors: INVALID_ARG
 * (operator, N_down or lattice mismatch, sector index), SYMMETRY (momentum
 * not K + Q). */
int qs3_sq_apply(int32_t op, qs3_basis_t src, int32_t s_src, const void *phi, qs3_basis_t dst, int32_t s_dst,
                 const int32_t *Q, void *psi, void *stream);

/* qs3_dsf for any S^alpha_q (op as in qs3_sq_apply): dst holds, in order,
 * the n_q sectors (N_down + dN, K + Q_n) with dN = -1, +1, 0 for S^+, S^-,
 * S^z.  The field enters the resolvent as the Zeeman shift h_field * dN
 * (poles at E_n - e0 + h_field dN).  subtract_trivial != 0 with op = S^z
 * removes, at every q equivalent to 0, the ground state's own delta peak
 * broadened to eta / (pi (omega^2 + eta^2)) M^2 / N with M = N/2 - N_down
 * (the paper's longitudinal factor with the trivial component subtracted).
 * Other arguments, outputs and errors as qs3_dsf. */
int qs3_dsf_op(int32_t op, int32_t subtract_trivial, qs3_basis_t src, int32_t s_src, const void *gs, double e0,
               qs3_basis_t dst, int32_t n_q, const int32_t *Q, int32_t n_iter, double eta, double h_field,
               int32_t n_omega, const double *omega, double *s_qw, double *alpha, double *beta, double *norm2,
               void *stream);

/* Full diagonalisation of sector s of b (Sec. "Full diagonalization", the
 * paper's ALG = 3): the dense Hermitian block of H in the sector's basis is
 * assembled column by column from H Phi on unit vectors (only sector s
 * active) and diagonalised by a library dense eigensolver (cuSOLVER zheevd).
 * evals: host, dims[s] doubles, ascending.  evecs: NULL, or a caller-owned
 * device C128 array of dims[s]^2 elements that receives the eigenvectors as
 * columns (column-major, eigenvector nu at evecs + nu * dims[s]).  Limit:
 * dims[s] <= 16384 (INVALID_ARG beyond); the call allocates the d^2 matrix
 * when evecs is NULL (OOM if it does not fit) and synchronises stream.
 * NOT_CONVERGED if the eigensolver reports failure. */
int qs3_full_diag(qs3_basis_t b, int32_t s, double *evals, void *evecs, void *stream);

/* Thermal averages of Eq. (ens) over a list of levels E_nu (host arrays of
 * n_levels; the levels of all sectors wanted, e.g. from qs3_full_diag):
 * log_z[k] = log sum_nu m_nu e^{-beta_k E_nu} and avg[k] = sum_nu m_nu
 * e^{-beta_k E_nu} A_nu / Z(beta_k), with A = E when A is NULL and m = 1 when
 * mult is NULL.  Exponents are shifted by the lowest level, so large beta
 * does not underflow.  Host arithmetic; log_z or avg may be NULL.
 * INVALID_ARG for an empty list, a non-finite level or a negative weight. */
int qs3_thermal(int64_t n_levels, const double *E, const double *A, const double *mult, int32_t n_beta,
                const double *beta, double *log_z, double *avg);

/* Measured throughput of this GPU's arithmetic pipes (no counterpart in the
 * paper: the denominators of the ALU rooflines of the benchmark).  Each probe
 * runs 8 blocks of 256 threads per SM, every thread 8 independent chains of
 * one instruction kind, timed with CUDA events on stream (second of two
 * launches, about 10-30 ms each):
 *   fp64_fma_per_s  fp64 fused multiply-adds per second (thread operations),
 *   fp32_fma_per_s  fp32 fused multiply-adds per second,
 *   int_mad_per_s   32-bit integer multiply-adds per second,
 *   int_alu_per_s   32-bit integer xor / add operations per second,
 *   issue_per_s     warp instructions per second of the fp32 probe (one
 *                   instruction per 32 lanes; a lower bound of the issue rate),
 *   n_sms           multiprocessors of the current device.
 * Errors: INVALID_ARG (NULL out), OOM, CUDA.  Synchronises stream. */
typedef struct {
    double fp64_fma_per_s, fp32_fma_per_s, int_mad_per_s, int_alu_per_s, issue_per_s;
    int32_t n_sms, reserved;
} qs3_peaks;
int qs3_probe_peaks(qs3_peaks *out, void *stream);

/* Allocation fault injection for tests of the error paths (no counterpart
 * in the paper).  after >= 0: the next `after` device allocations of the
 * library succeed as usual, every later one fails with QS3_ERR_OOM without
 * calling the CUDA allocator, until the next call; after < 0 switches the
 * injection off.  Process-wide (all threads).  Returns the previous setting
 * (-1 = off).  Calls that fail this way release what they allocated. */
int64_t qs3_inject_alloc_failure(int64_t after);

/* Wait-timeout injection for tests of the bounded device waits (no
 * counterpart in the paper).  n > 0: the next n launches of the copy-ring
 * dot pass (k_dotb) run with their copy warp issuing no copies, so every
 * consumer warp's wait on its first stage runs out after one second and the
 * call that launched it returns QS3_ERR_TIMEOUT (the context stays usable;
 * no fault, trap or endless wait is involved).  n <= 0 switches it off.
 * Process-wide.  Returns the previous count. */
int32_t qs3_inject_wait_timeout(int32_t n);

/* Text of a status code, and of the last failure on the calling thread. */
const char *qs3_strerror(int status);
const char *qs3_last_error(void);

/* Library version string. */
const char *qs3_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (library primitives such as the CUB sort are not counted). */
uint64_t qs3_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* QS3_H */
