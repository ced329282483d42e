/* nucleus_debug.h -- fault injection for tests of libnucleus's error paths.
 *
 * Host-side settings only (process-wide, not thread-safe; set them between calls).  Nothing here
 * makes a GPU fault, trap or hang: a shortened wait limit makes the persistent kernels' bounded
 * grid barriers give up early, every block then leaves its loop and the call returns
 * NH_ERR_TIMEOUT with the context intact; a forced hash-table capacity makes the (bounded)
 * insertion run out of slots and the call returns NH_ERR_TABLE_FULL.  Status codes are those of
 * nucleus.h. */
#ifndef NUCLEUS_DEBUG_H
#define NUCLEUS_DEBUG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* wait limit, in ns, of the grid barriers of the peel (nh_peel_and_link, nh_approx_nucleus,
 * nh_hierarchy_enqueue) and of the two-phase / label hierarchies; 0 = the default (60 s) */
#define NH_INJECT_WAIT_NS 1
/* capacity, in slots (a power of two), of the edge table (nh_build_orientation) and of the
 * triangle table (nh_index_r_cliques, r = 3) built from now on; 0 = automatic (load <= 0.5) */
#define NH_INJECT_TABLE_CAP 2
/* value every s-clique-degree starts from before counting (nh_count_s_cliques and the counting
 * step of nh_hierarchy_enqueue, s >= 3) in place of 0, so that a small graph reaches the uint32
 * limit: counting then returns NH_ERR_COUNT_OVERFLOW; 0 = off */
#define NH_INJECT_COUNT_BASE 3

/* Set one injection.  value >= 0 (NH_INJECT_TABLE_CAP: 0 or a power of two; NH_INJECT_COUNT_BASE:
 * < 2^32).  Returns NH_OK or NH_ERR_INVALID (unknown `what`, bad value; nothing changed). */
int nh_debug_inject(int what, int64_t value);

/* Round trace of the persistent peel kernels (nh_peel_and_link, nh_approx_nucleus): when set, the
 * next peels write, for every round t = 1, 2, ... (while t <= cap), eight words at log[8 (t-1)]:
 * (frontier size << 32 | levels opened so far), the device global timer (ns) at the end of the
 * round, the out-list entries the (2,4) triangle-list re-listing expanded in the round,
 * (its sub-tasks << 32 | of which block sub-tasks), then block 0's timer when that re-listing
 * starts, after it split the round into sub-tasks, after its warp phase and at its end (0 for
 * the other re-listings).  log: device uint64[8 cap], owned by the caller and kept alive while
 * set; NULL or cap 0 turns the trace off.  Returns NH_OK or NH_ERR_INVALID (cap < 0). */
int nh_debug_round_log(uint64_t* log, int64_t cap);

#ifdef __cplusplus
}
#endif

#endif
