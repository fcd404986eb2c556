// qs3_solver.cu -- Lanczos / thick-restart Lanczos (placeholder entry points)
#include "qs3_internal.cuh"

extern "C" int qs3_lanczos(qs3_basis_t, const qs3_solve_opts *, double *, void *, qs3_solve_info *, void *) {
    return qs3::set_err(QS3_ERR_STATE, "not built yet");
}
extern "C" int qs3_trlanczos(qs3_basis_t, const qs3_solve_opts *, double *, void *, qs3_solve_info *, void *) {
    return qs3::set_err(QS3_ERR_STATE, "not built yet");
}
