// api.cu -- error reporting shared by the entry points of libpic.so.
#include <cstdarg>
#include <cstdio>

#include "pic_internal.cuh"

namespace pic {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

pic_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return PIC_ERR_CUDA;
}

}  // namespace pic

extern "C" const char* pic_last_error(void) { return pic::g_err; }

extern "C" const char* pic_version(void) { return "pic-gb300 0.1 (sm_103a)"; }
