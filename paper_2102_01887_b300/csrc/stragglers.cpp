// stragglers.cpp -- host-side detection of stragglers and failed invocations
// (Section 3.4, "Handling stragglers and invocation failures"; the time-out of
// Section 5).  The Scheduler tracks every invocation's execution time; an
// invocation that reports an error, or that runs past its time-out, gets a
// duplicate invocation, which goes back through slack allotment (Algorithm 1)
// and configuration (Eq. 1) at the time the failure is seen -- with less of
// the pipeline's target left, so with less slack.  Host code only: nothing
// here touches the GPU; the duplicates are scheduled by the normal entry
// points.
#include <cstdint>

#include "../../include/llama.h"

extern "C" int llama_stragglers(int64_t n, const llama_decision *dec, const int64_t *obs_us, const uint8_t *failed,
                                int64_t now_us, int32_t timeout_num, int32_t timeout_den, int64_t tick_us,
                                int64_t *dup_idx, int64_t *resubmit_us, int64_t *n_dup) {
    if (n < 0 || !n_dup || timeout_num < 1 || timeout_den < 1 || tick_us < 1) return LLAMA_EINVAL;
    if (n > 0 && (!dec || !obs_us || !dup_idx || !resubmit_us)) return LLAMA_EINVAL;
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        const llama_decision &d = dec[i];
        if (d.cfg < 0) continue;  // not decided: nothing was started
        if (obs_us[i] < 0) return LLAMA_EINVAL;
        // time-out: ceil(timeout_num * L / timeout_den) microseconds after the start
        // (L < 2^31, timeout_num < 2^31: the product fits in 64 bits)
        const int64_t limit = ((int64_t)timeout_num * d.lat + timeout_den - 1) / timeout_den;
        const bool err = failed && failed[i];
        int64_t seen;  // when the Scheduler learns of it, after the invocation started at now_us
        if (err && obs_us[i] <= limit) seen = obs_us[i];  // the error arrives before the time-out
        else if (obs_us[i] > limit) seen = limit;          // still running at the time-out
        else continue;                                     // completed in time
        // the Manager checks at its ticks: the first tick at or after the event
        const int64_t t = now_us + seen;
        dup_idx[k] = i;
        resubmit_us[k] = (t + tick_us - 1) / tick_us * tick_us;
        ++k;
    }
    *n_dup = k;
    return LLAMA_OK;
}
