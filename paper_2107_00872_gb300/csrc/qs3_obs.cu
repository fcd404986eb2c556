// qs3_obs.cu -- observables (placeholder entry points)
#include "qs3_internal.cuh"

extern "C" int qs3_correlations(qs3_basis_t, int32_t, const void *, int32_t, const int32_t *, double *, double *,
                                double *, int32_t, const double *, double *, double *, void *) {
    return qs3::set_err(QS3_ERR_STATE, "not built yet");
}
extern "C" int qs3_smq(qs3_basis_t, int32_t, const void *, qs3_basis_t, int32_t, const int32_t *, void *, void *) {
    return qs3::set_err(QS3_ERR_STATE, "not built yet");
}
extern "C" int qs3_dsf(qs3_basis_t, int32_t, const void *, double, qs3_basis_t, int32_t, const int32_t *, int32_t,
                       double, double, int32_t, const double *, double *, double *, double *, double *, void *) {
    return qs3::set_err(QS3_ERR_STATE, "not built yet");
}
