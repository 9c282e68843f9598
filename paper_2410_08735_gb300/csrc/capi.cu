// Status strings, thread-local error detail and version of the C ABI (include/rte.h).
#include <string>

#include "internal.h"

#include <atomic>

namespace rte {
static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
void set_error(const std::string& msg) { g_last_error = msg; }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(); }
}  // namespace rte

extern "C" {

const char* rte_status_string(int status) {
  switch (status) {
    case RTE_OK: return "RTE_OK";
    case RTE_ERR_INVALID_ARG: return "RTE_ERR_INVALID_ARG";
    case RTE_ERR_CUDA: return "RTE_ERR_CUDA";
    case RTE_ERR_OOM: return "RTE_ERR_OOM";
    case RTE_ERR_NOT_CONVERGED: return "RTE_ERR_NOT_CONVERGED";
    case RTE_ERR_NUMERIC: return "RTE_ERR_NUMERIC";
    case RTE_ERR_TIMEOUT: return "RTE_ERR_TIMEOUT";
    case RTE_ERR_UNSUPPORTED: return "RTE_ERR_UNSUPPORTED";
    case RTE_ERR_IO: return "RTE_ERR_IO";
    default: return "RTE_ERR_UNKNOWN";
  }
}

const char* rte_last_error(void) { return rte::g_last_error.c_str(); }

long long rte_kernel_launches(void) { return rte::g_launches.load(); }

int rte_version(int* major, int* minor) {
  if (major) *major = 0;
  if (minor) *minor = 1;
  return RTE_OK;
}

}  // extern "C"
