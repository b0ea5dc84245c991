// status.h -- thread-local host error text for the C ABI.
#pragma once
#include <stdarg.h>

// Records a formatted message for gp_error_string() and returns `code`.
int gp_fail(int code, const char* fmt, ...);
// Clears the message at the start of an entry point.
void gp_clear_error();
