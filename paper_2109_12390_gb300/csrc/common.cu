// Thread-local error message behind mpm_last_error().
#include <string>

#include "common.cuh"

namespace mpmrom {
namespace {
thread_local std::string g_last_error;
}
mpm_status set_error(mpm_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
}  // namespace mpmrom

extern "C" const char* mpm_last_error(void) { return mpmrom::g_last_error.c_str(); }
