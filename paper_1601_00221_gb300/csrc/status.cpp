// status.cpp -- thread-local host error text for the C ABI.
#include "status.h"

#include <stdio.h>

#include "../../include/gpeval.h"

namespace {
thread_local char g_msg[512] = "";
}

int gp_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return code;
}

void gp_clear_error() { g_msg[0] = '\0'; }

extern "C" const char* gp_error_string(void) { return g_msg; }

extern "C" int32_t gp_version(void) { return 10000; }
