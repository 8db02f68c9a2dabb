// Library-wide entry points: version string and per-thread error messages.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

#include <atomic>

namespace sbr {
namespace {
thread_local char g_err[512] = "";
std::atomic<unsigned long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
}  // namespace sbr

extern "C" const char* sbr_version(void) { return "libsbr 0.1 (sm_103a)"; }

extern "C" void sbr_last_error(char* buf, size_t n) {
  if (!buf || n == 0) return;
  strncpy(buf, sbr::g_err, n - 1);
  buf[n - 1] = '\0';
}

extern "C" uint64_t sbr_launch_count(void) { return sbr::g_launches.load(std::memory_order_relaxed); }
