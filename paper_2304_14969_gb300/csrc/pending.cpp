// Entry points whose implementation is not part of this build yet: they
// validate nothing and report QSIM_E_UNSUPPORTED.
#include "qsim_internal.h"

using namespace qs;

extern "C" {

qsim_status qsim_batch_create(const qsim_circuit *const *, int, const qsim_batch_opts *, qsim_batch **out)
{
    if (out) *out = nullptr;
    return fail(QSIM_E_UNSUPPORTED, "batched runs are not available in this build");
}
qsim_status qsim_batch_destroy(qsim_batch *) { return QSIM_OK; }
qsim_status qsim_batch_upload(qsim_batch *, int, const void *) { return fail(QSIM_E_UNSUPPORTED, "no batches"); }
qsim_status qsim_batch_reset(qsim_batch *) { return fail(QSIM_E_UNSUPPORTED, "no batches"); }
qsim_status qsim_batch_run(qsim_batch *, double *, double *) { return fail(QSIM_E_UNSUPPORTED, "no batches"); }
qsim_status qsim_batch_download(qsim_batch *, int, void *) { return fail(QSIM_E_UNSUPPORTED, "no batches"); }
qsim_status qsim_batch_info(const qsim_batch *, int64_t *) { return fail(QSIM_E_UNSUPPORTED, "no batches"); }
qsim_status qsim_autotune(const qsim_circuit *, qsim_dtype, const char *, qsim_run_opts *, double *)
{
    return fail(QSIM_E_UNSUPPORTED, "autotuner is not available in this build");
}

}  // extern "C"
