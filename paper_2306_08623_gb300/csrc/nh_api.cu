// nh_api.cu -- status strings and version of the C-ABI (the entry points live beside their kernels).
#include <atomic>

#include "nh_internal.cuh"
#include "nucleus_debug.h"

static std::atomic<long long> g_launches{0};

void nh_note_launch(int64_t k) { g_launches.fetch_add((long long)k, std::memory_order_relaxed); }

extern "C" int64_t nh_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

extern "C" const char* nh_status_string(int status) {
  switch (status) {
    case NH_OK: return "ok";
    case NH_ERR_INVALID: return "invalid argument";
    case NH_ERR_OOM: return "device allocation failed";
    case NH_ERR_TABLE_FULL: return "r-clique hash table full";
    case NH_ERR_OVERFLOW: return "device work queue overflow";
    case NH_ERR_TIMEOUT: return "bounded device wait expired";
    case NH_ERR_UNSUPPORTED: return "unsupported (r,s) or device";
    case NH_ERR_CUDA: return "CUDA runtime error";
    case NH_ERR_INTERNAL: return "device consistency check failed";
    case NH_ERR_COUNT_OVERFLOW: return "s-clique-degree exceeds 2^32 - 1";
    default: return "unknown status";
  }
}

extern "C" int nh_version(void) { return 100; }

// fault injection (include/nucleus_debug.h); read by the drivers in nh_peel.cu and nh_orient.cu
long long g_nh_inject_wait_ns = 0;
long long g_nh_inject_table_cap = 0;
long long g_nh_inject_count_base = 0;

extern "C" int nh_debug_inject(int what, int64_t value) {
  if (value < 0) return NH_ERR_INVALID;
  if (what == NH_INJECT_WAIT_NS) {
    g_nh_inject_wait_ns = (long long)value;
    return NH_OK;
  }
  if (what == NH_INJECT_TABLE_CAP) {
    if (value != 0 && (value & (value - 1))) return NH_ERR_INVALID;
    g_nh_inject_table_cap = (long long)value;
    return NH_OK;
  }
  if (what == NH_INJECT_COUNT_BASE) {
    if (value > 0xffffffffll) return NH_ERR_INVALID;
    g_nh_inject_count_base = (long long)value;
    return NH_OK;
  }
  return NH_ERR_INVALID;
}

// round trace (include/nucleus_debug.h); read by the peel driver in nh_peel.cu
uint64_t* g_nh_round_log = nullptr;
long long g_nh_round_log_cap = 0;

extern "C" int nh_debug_round_log(uint64_t* log, int64_t cap) {
  if (cap < 0) return NH_ERR_INVALID;
  g_nh_round_log = (cap > 0) ? log : nullptr;
  g_nh_round_log_cap = (log != nullptr) ? (long long)cap : 0;
  return NH_OK;
}
