/* abi_layout.c -- prints the size and the field offsets of every struct of
 * include/szgb.h, one "struct.field offset" line each, for the test that
 * compares them with the Python binding's ctypes mirrors. */
#include <stddef.h>
#include <stdio.h>

#include "../../include/szgb.h"

#define F(S, f) printf(#S "." #f " %zu\n", offsetof(S, f))
#define Z(S) printf(#S ".sizeof %zu\n", sizeof(S))

int main(void) {
    Z(szgb_params);
    F(szgb_params, ndim); F(szgb_params, shape); F(szgb_params, mode); F(szgb_params, eb_abs);
    F(szgb_params, eb_rel); F(szgb_params, layers); F(szgb_params, m); F(szgb_params, theta);
    F(szgb_params, variant); F(szgb_params, chunk_points);
    Z(szgb_stats);
    F(szgb_stats, n_points); F(szgb_stats, n_unpred); F(szgb_stats, stream_bytes); F(szgb_stats, m);
    F(szgb_stats, maxlen); F(szgb_stats, nsym); F(szgb_stats, eb_f); F(szgb_stats, xmin); F(szgb_stats, xmax);
    F(szgb_stats, status);
    Z(szgb_quality);
    F(szgb_quality, max_abs_err); F(szgb_quality, max_rel_err); F(szgb_quality, rmse); F(szgb_quality, nrmse);
    F(szgb_quality, psnr); F(szgb_quality, pearson); F(szgb_quality, x_min); F(szgb_quality, x_max);
    F(szgb_quality, n);
    Z(szgb_request);
    F(szgb_request, op); F(szgb_request, in); F(szgb_request, in_bytes); F(szgb_request, params);
    F(szgb_request, out); F(szgb_request, out_cap);
    return 0;
}
