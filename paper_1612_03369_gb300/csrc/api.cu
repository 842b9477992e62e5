// api.cu -- error reporting shared by the entry points of libpic.so.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>

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

static std::atomic<unsigned long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

}  // namespace pic

using namespace pic;

extern "C" uint64_t pic_kernel_launches(void) { return (uint64_t)g_launches.load(); }

extern "C" pic_status pic_timing_enable(pic_particles p, int on) {
  if (!p) return (set_error("pic_timing_enable: null handle"), PIC_ERR_ARG);
  p->timing = on ? 1 : 0;
  return PIC_OK;
}

extern "C" pic_status pic_set_advect_staging(pic_particles p, int on) {
  if (!p) return (set_error("pic_set_advect_staging: null handle"), PIC_ERR_ARG);
  p->stage_cells = on ? 1 : 0;
  return PIC_OK;
}

extern "C" pic_status pic_timing_read(pic_particles p, double* advect_ms, double* rebin_ms, uint64_t* steps) {
  if (!p) return (set_error("pic_timing_read: null handle"), PIC_ERR_ARG);
  double a = 0.0, r = 0.0;
  for (int k = 0; k < p->n_ev; ++k) {
    cudaEvent_t* e = p->ev + 3 * k;
    PIC_CUDA(cudaEventSynchronize(e[2]));
    float t1 = 0.f, t2 = 0.f;
    PIC_CUDA(cudaEventElapsedTime(&t1, e[0], e[1]));
    PIC_CUDA(cudaEventElapsedTime(&t2, e[1], e[2]));
    a += t1;
    r += t2;
  }
  if (advect_ms) *advect_ms = a;
  if (rebin_ms) *rebin_ms = r;
  if (steps) *steps = (uint64_t)p->n_ev;
  p->n_ev = 0;
  return PIC_OK;
}

extern "C" const char* pic_last_error(void) { return pic::g_err; }

extern "C" const char* pic_version(void) { return "pic-gb300 0.1 (sm_103a)"; }
