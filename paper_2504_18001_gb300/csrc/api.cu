// Error reporting and version of the C ABI.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "cinr_internal.cuh"

namespace cinr {

static thread_local char g_last_error[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  return set_error(CINR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace cinr

extern "C" int cinr_last_error(char* buf, size_t n) {
  if (buf && n > 0) {
    strncpy(buf, cinr::g_last_error, n - 1);
    buf[n - 1] = '\0';
  }
  return CINR_OK;
}

extern "C" int cinr_version(void) { return 100; }

extern "C" int cinr_device_checks(void) { return CINR_CHECK ? 1 : 0; }
