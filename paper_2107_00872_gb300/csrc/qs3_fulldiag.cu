// qs3_fulldiag.cu -- full diagonalisation of one symmetry sector (Sec.
// "Full diagonalization") and the thermal averages of Eq. (ens).
//
// The dense Hermitian block of H in a sector's basis is assembled column by
// column from the matrix-free product itself: column j = H e_j, with only the
// sector's rows active, so every matrix element comes from the same code as
// H Phi.  A library dense eigensolver (cuSOLVER zheevd, the counterpart of
// the paper's LAPACK ZHEEVR) gives all eigenvalues and, on request, the
// eigenvectors.  The paper notes the matrix dimension is practical up to
// O(10^4); the entry point accepts at most FULL_DIAG_MAX rows.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "qs3_internal.cuh"

namespace qs3 {

constexpr int FULL_DIAG_MAX = 16384;

__global__ void k_set_entry(double2 *x, uint64_t i, double2 v) { x[i] = v; }

static int full_diag(Basis &B, int s, double *evals, double2 *evecs, cudaStream_t st) {
    if (s < 0 || s >= B.S) return set_err(QS3_ERR_INVALID_ARG, "sector index %d", s);
    const uint64_t d = B.dims[s];
    if (d == 0) return QS3_OK;
    if (d > (uint64_t)FULL_DIAG_MAX)
        return set_err(QS3_ERR_INVALID_ARG, "sector dimension %llu above the full-diagonalisation limit %d",
                       (unsigned long long)d, FULL_DIAG_MAX);
    const int n = (int)d;
    DevBuf own, x, y, act, w;
    double2 *A = evecs;
    if (!A) {
        QS3_TRY(own.alloc(d * d * sizeof(double2)));
        A = own.as<double2>();
    }
    QS3_TRY(x.alloc(B.total * sizeof(double2)));
    QS3_TRY(y.alloc(B.total * sizeof(double2)));
    QS3_TRY(w.alloc(d * sizeof(double)));
    std::vector<int> mask(B.S, 0);
    mask[s] = 1;
    QS3_TRY(act.upload(mask.data(), mask.size() * sizeof(int)));
    QS3_CUDA(cudaMemsetAsync(x.p, 0, B.total * sizeof(double2), st));
    const uint64_t off = B.offs[s];
    const qs3_dtype dt = QS3_C128;
    for (uint64_t j = 0; j < d; ++j) {
        k_set_entry<<<1, 1, 0, st>>>(x.as<double2>(), off + j, make_double2(1.0, 0.0));
        QS3_LAUNCHED();
        QS3_TRY(hphi_launch(B, dt, x.p, y.p, st, act.as<int>()));
        k_set_entry<<<1, 1, 0, st>>>(x.as<double2>(), off + j, make_double2(0.0, 0.0));
        QS3_LAUNCHED();
        QS3_CUDA(cudaMemcpyAsync(A + j * d, y.as<double2>() + off, d * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return set_err(QS3_ERR_CUDA, "cusolverDnCreate failed");
    int rc = QS3_OK;
    int lwork = 0;
    DevBuf work, info;
    if (cusolverDnSetStream(h, st) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnZheevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, (cuDoubleComplex *)A, n,
                                    w.as<double>(), &lwork) != CUSOLVER_STATUS_SUCCESS) {
        rc = set_err(QS3_ERR_CUDA, "cusolver workspace query failed");
    }
    if (rc == QS3_OK) rc = work.alloc((size_t)std::max(lwork, 1) * sizeof(cuDoubleComplex));
    if (rc == QS3_OK) rc = info.alloc(sizeof(int));
    if (rc == QS3_OK &&
        cusolverDnZheevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, (cuDoubleComplex *)A, n,
                         w.as<double>(), work.as<cuDoubleComplex>(), lwork, info.as<int>()) != CUSOLVER_STATUS_SUCCESS)
        rc = set_err(QS3_ERR_CUDA, "cusolverDnZheevd failed");
    int hinfo = 0;
    if (rc == QS3_OK) {
        if (cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(evals, w.p, d * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = set_err(QS3_ERR_CUDA, "copy of the eigenvalues failed");
        else if (hinfo != 0)
            rc = set_err(QS3_ERR_NOT_CONVERGED, "zheevd info %d", hinfo);
    }
    cusolverDnDestroy(h);
    return rc;
}

// Eq. (ens) over a list of levels, shifted by the lowest level
static void thermal(int64_t n, const double *E, const double *A, const double *mult, int nb, const double *beta,
                    double *logz, double *avg) {
    double e0 = E[0];
    for (int64_t i = 1; i < n; ++i) e0 = std::min(e0, E[i]);
    for (int k = 0; k < nb; ++k) {
        double z = 0.0, za = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double wgt = (mult ? mult[i] : 1.0) * std::exp(-beta[k] * (E[i] - e0));
            z += wgt;
            za += wgt * (A ? A[i] : E[i]);
        }
        if (logz) logz[k] = std::log(z) - beta[k] * e0;
        if (avg) avg[k] = za / z;
    }
}

}  // namespace qs3

using namespace qs3;

extern "C" int qs3_full_diag(qs3_basis_t b, int32_t s, double *evals, void *evecs, void *stream) {
    clear_err();
    if (!b || !evals) return set_err(QS3_ERR_INVALID_ARG, "NULL argument");
    return full_diag(b->B, s, evals, (double2 *)evecs, (cudaStream_t)stream);
}

extern "C" int qs3_thermal(int64_t n_levels, const double *E, const double *A, const double *mult, int32_t n_beta,
                           const double *beta, double *log_z, double *avg) {
    clear_err();
    if (n_levels < 1 || !E || n_beta < 0 || (n_beta > 0 && !beta)) return set_err(QS3_ERR_INVALID_ARG, "bad argument");
    for (int64_t i = 0; i < n_levels; ++i)
        if (!std::isfinite(E[i]) || (mult && !(mult[i] >= 0.0))) return set_err(QS3_ERR_INVALID_ARG, "level %lld", (long long)i);
    thermal(n_levels, E, A, mult, n_beta, beta, log_z, avg);
    return QS3_OK;
}
