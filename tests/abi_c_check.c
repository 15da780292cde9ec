/* A plain C99 client of the library's C ABI (include/mbd_gb300.h, include/mbd_gb300_kernels.h),
 * built with -std=c99 -pedantic -Werror by tests/test_abi_c.py and run without a GPU: it
 * prints the layout of the option and profile structs as a C compiler sees them, the
 * defaults the library fills in, and the codes of calls that must fail before any device
 * work (invalid options, NULL handles and pointers). */
#include <stddef.h>
#include <stdio.h>

#include "mbd_gb300.h"
#include "mbd_gb300_kernels.h"

#define FIELD(T, f) printf("offset %s %s %lu\n", #T, #f, (unsigned long)offsetof(T, f))

int main(void) {
    mbd_options opt;
    mbd_ctx *ctx = NULL;
    int code = -1;
    char origin[64], msg[128];
    double e = 0.0;
    long long count = 0;

    printf("sizeof mbd_options %lu\n", (unsigned long)sizeof(mbd_options));
    FIELD(mbd_options, n_freq);
    FIELD(mbd_options, beta);
    FIELD(mbd_options, a);
    FIELD(mbd_options, precision);
    FIELD(mbd_options, ns_tol);
    FIELD(mbd_options, ns_max_iter);
    FIELD(mbd_options, tc_chunk_stages);
    FIELD(mbd_options, ewald_gamma);
    FIELD(mbd_options, real_cutoff);
    FIELD(mbd_options, recip_cutoff);
    FIELD(mbd_options, scs_mode);
    FIELD(mbd_options, learned_max_error);
    FIELD(mbd_options, mixed_max_error);
    FIELD(mbd_options, learned_estimate_scale);
    printf("sizeof mbd_profile %lu\n", (unsigned long)sizeof(mbd_profile));
    FIELD(mbd_profile, launches);
    FIELD(mbd_profile, gemm_launches);
    FIELD(mbd_profile, gemm_ms);
    FIELD(mbd_profile, gemm_flops);
    FIELD(mbd_profile, screening_ms);
    FIELD(mbd_profile, screening_flops);
    FIELD(mbd_profile, newton_schulz_ms);
    FIELD(mbd_profile, gradient_ms);
    FIELD(mbd_profile, total_ms);
    FIELD(mbd_profile, tc_launches);
    FIELD(mbd_profile, tc_ms);
    FIELD(mbd_profile, tc_flops);
    FIELD(mbd_profile, correction_ms);

    printf("rc default_options %d\n", mbd_default_options(&opt));
    printf("default n_freq %d beta %.17g a %.17g precision %d ns_tol %.17g ns_max_iter %d "
           "tc_chunk_stages %d scs_mode %d learned_max_error %.17g mixed_max_error %.17g "
           "learned_estimate_scale %.17g\n",
           opt.n_freq, opt.beta, opt.a, opt.precision, opt.ns_tol, opt.ns_max_iter, opt.tc_chunk_stages,
           opt.scs_mode, opt.learned_max_error, opt.mixed_max_error, opt.learned_estimate_scale);
    printf("rc default_options_null %d\n", mbd_default_options(NULL));

    opt.n_freq = 0;   /* rejected before the device is touched */
    printf("rc create_bad_n_freq %d\n", mbd_create(&ctx, 0, &opt));
    printf("ctx_after_failed_create %s\n", ctx == NULL ? "null" : "set");
    printf("rc create_null_out %d\n", mbd_create(NULL, 0, NULL));
    printf("rc destroy_null %d\n", mbd_destroy(NULL));
    printf("rc evaluate_null %d\n", mbd_evaluate(NULL, &e, NULL, NULL, NULL, NULL));
    printf("rc evaluation_count_null %d\n", mbd_get_evaluation_count(NULL, &count));
    printf("rc exception_null %d\n", mbd_get_exception(NULL, &code, origin, msg, sizeof msg));
    printf("split_work_bytes %lu\n", (unsigned long)mbdk_gemm_f64_split_work_bytes(128, 256, 64));
    return 0;
}
