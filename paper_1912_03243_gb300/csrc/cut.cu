// Decomposition of entangling gates across a partition (Sec. 4, Eq. 2-3).
#include "plan.h"

using namespace sv;

extern "C" sv_status sv_cut_amplitudes(const char *text, int n, uint64_t maskA, int form, size_t m, const uint64_t *z,
                                       double *out, int *n_cut_out, void *stream) {
    (void)text; (void)n; (void)maskA; (void)form; (void)m; (void)z; (void)out; (void)n_cut_out; (void)stream;
    set_error("sv_cut_amplitudes is not available yet");
    return SV_ERR_UNSUPPORTED;
}
