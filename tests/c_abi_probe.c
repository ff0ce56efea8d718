/* A plain C99 client of libsv: the header compiles as C and the host-only
 * calls (no GPU needed) link and run.  Prints one line per check. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "sv.h"

int main(void) {
    /* complex64 at 20 qubits: 2^20 x 8 bytes; the two-byte code: codes plus scales */
    printf("bytes_c64_20 %zu\n", sv_bytes_required(20, SV_C64));
    printf("bytes_enc_20 %zu\n", sv_bytes_required(20, SV_ENC2B));
    double h[8];
    const int k = sv_gate_matrix("H", NULL, 0, h);
    printf("gate_H %d %.17g %.17g\n", k, h[0], h[6]);
    int64_t gates = 0, passes = 0, segments = 0;
    const char *text = "qubits 14\nH 0\nH 13\nCZ 0 13\nT 7\n";
    const sv_status s = sv_plan_stats(text, 14, SV_C64, 0, &gates, &passes, &segments);
    printf("plan %d %lld %lld\n", (int)s, (long long)gates, (long long)passes);
    const sv_status bad = sv_plan_stats("qubits 14\nH 99\n", 14, SV_C64, 0, &gates, &passes, &segments);
    printf("bad %d %s\n", (int)bad, strlen(sv_last_error()) > 0 ? "message" : "empty");
    return 0;
}
