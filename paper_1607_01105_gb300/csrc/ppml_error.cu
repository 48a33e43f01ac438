// Thread-local error reporting of the C ABI (ppml_last_error).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/ppml.h"
#include "ppml_internal.h"

namespace {
thread_local char g_msg[512] = {0};
}

int ppml_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

void ppml_clear_error() { g_msg[0] = 0; }

int ppml_check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ppml_fail(PPML_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return PPML_OK;
}

extern "C" const char* ppml_last_error(void) { return g_msg; }
