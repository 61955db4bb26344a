/* A plain C99 client of libespp_gb.so: it compiles against include/espp.h
 * alone and calls the library with no C++ or Python in between.
 *
 * Without a GPU it checks the host-only Hilbert ranks, an argument refusal,
 * and that creating a system reports the missing device as an error with a
 * message.  With a GPU it also places two WCA beads one sigma apart and
 * checks the pair force, 24 epsilon / sigma (WCA and LJ share their force
 * below 2^(1/6) sigma), and Newton's third law.  Exit status 0 on success. */
#include <stdint.h>
#include <stdio.h>

#include "espp.h"

int main(void) {
    int32_t rank[60];
    int seen[60] = {0};
    if (espp_hilbert_ranks(3, 4, 5, rank) != ESPP_OK) return 1;
    for (int k = 0; k < 60; ++k) {
        if (rank[k] < 0 || rank[k] >= 60 || seen[rank[k]]++) return 2;
    }

    const double box[3] = {10.0, 10.0, 10.0};
    espp_h h = NULL;
    if (espp_system_create(box, -1, NULL, 0, NULL, ESPP_FP64, 1, NULL, &h) != ESPP_ERR_ARG) return 3;

    int rc = espp_system_create(box, 2, NULL, 0, NULL, ESPP_FP64, 7, NULL, &h);
    if (rc != ESPP_OK) {
        const char* msg = espp_last_error(NULL);
        printf("create refused: %d (%s)\n", rc, msg ? msg : "");
        return (rc < 0 && msg && msg[0]) ? 0 : 4;
    }
    const double wca[2] = {1.0, 1.0};
    const double x[6] = {4.5, 5.0, 5.0, 5.5, 5.0, 5.0};
    double f[6] = {0};
    if (espp_set_interaction(h, ESPP_WCA, 0, 0, wca, 2) != ESPP_OK) return 5;
    if (espp_set_state(h, x, NULL, NULL, ESPP_HOST) != ESPP_OK) return 6;
    if (espp_build_neighbors(h, 1.122462048309373, 0.4) != ESPP_OK) return 7;
    if (espp_compute_forces(h, f, ESPP_HOST) != ESPP_OK) return 8;
    espp_system_destroy(h);
    const double e0 = f[0] + 24.0, e3 = f[3] - 24.0;
    if (e0 * e0 > 1e-20 || e3 * e3 > 1e-20) return 9;
    if (f[1] != 0.0 || f[2] != 0.0 || f[0] + f[3] != 0.0) return 10;
    printf("ok\n");
    return 0;
}
