/*
 * lbf_debug.h - test hooks of the index-checked build of the library (liblbf_debug.so, compiled
 * with LBF_DEBUG). The release library liblbf.so does not export these symbols.
 */
#ifndef LBF_DEBUG_H
#define LBF_DEBUG_H

#include "lbf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Exercises the give-up path of the bounded mbarrier wait that guards every TMA plane load of the
   fused step, without any copy in flight: one CTA initialises an mbarrier that nothing ever
   arrives on, waits on it with the same bounded wait as the fused step but with a limit of
   `polls` polls, and when the wait gives up sets the same error bit of the context's flags that
   the fused step sets (a plane load that did not complete in time). The next lbf_synchronize then
   returns LBF_EINTERNAL. polls: 1 .. 2^20 (LBF_EINVAL otherwise). Asynchronous on the context's
   stream; the context stays usable after lbf_synchronize reported the error once.
   Paper: no counterpart (failure detection of the library's own waits). */
lbf_status lbf_debug_wait_probe(lbf_ctx* ctx, unsigned polls);

#ifdef __cplusplus
}
#endif

#endif /* LBF_DEBUG_H */
