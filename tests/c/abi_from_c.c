/* A plain C99 caller of the library: includes the public header, links
 * libigapw.so and exercises the argument checks of igapw_create, which return
 * before any CUDA call (so this runs on a machine without a GPU).  Prints one
 * line per call: return code, whether *out was cleared, the error text. */
#include <stdio.h>
#include <string.h>

#include "igapw.h"

static void report(const char* what, int rc, igapw_ctx* ctx) {
    printf("%s %d %d %s\n", what, rc, ctx == NULL, igapw_last_error(NULL));
}

int main(void) {
    igapw_desc d;
    igapw_ctx* ctx = NULL;
    int rc;
    memset(&d, 0, sizeof d);
    d.dim = 4;
    rc = igapw_create(&ctx, &d, NULL);
    report("dim", rc, ctx);
    d.dim = 2;
    d.n_elem[0] = d.n_elem[1] = 4;
    d.degree = 1;
    d.nq = 3;
    rc = igapw_create(&ctx, &d, NULL);
    report("degree", rc, ctx);
    rc = igapw_create(&ctx, NULL, NULL);
    report("desc", rc, ctx);
    rc = igapw_create(NULL, &d, NULL);
    report("out", rc, ctx);
    return 0;
}
