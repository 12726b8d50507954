// Library-wide helpers behind the C ABI: per-thread error text, version,
// device properties.
#include <cstdarg>

#include "ss_internal.cuh"

namespace ss {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace ss

extern "C" const char* ss_last_error(void) { return ss::g_err; }

extern "C" const char* ss_version(void) { return "sparse-spectral-gb300 0.1 (sm_103a)"; }
