// Reduced density matrices of a state on the alpha x beta subspace.
#include "sqd_internal.cuh"

int launch_rdm(sqd_ctx *ctx, const sqd_tables *t, const double *C, double *rdm1, double *rdm2) {
    (void)t; (void)C; (void)rdm1; (void)rdm2;
    return sqd_fail(ctx, SQD_EINVAL, "sqd_rdm is not available in this build");
}
