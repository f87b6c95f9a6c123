// Error reporting and version of the C ABI.
#include <string>

#include "common.cuh"

namespace mcd {
static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }
}  // namespace mcd

extern "C" const char *mcd_last_error(void) { return mcd::g_last_error.c_str(); }

extern "C" const char *mcd_version(void) { return "mcd-gb300 0.1 (sm_103a)"; }
