/*
 * Host-side test program for the C ABI of include/pcc.h, linked either
 * against libpcc.so itself or against a copy of the library whose host code
 * is built with AddressSanitizer and UndefinedBehaviorSanitizer (then any
 * sanitizer report fails the run).  It needs no GPU: every call here must be
 * rejected by the library's own argument checks, before any CUDA work, with
 * the documented error code and a message in pcc_last_error().  A device
 * index that does not exist must fail in pcc_create with the output left
 * NULL.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pcc.h"

static int failures = 0;

/* rc must equal `want` and leave a non-empty message naming the call. */
static void expect(int rc, int want, const char *call)
{
    const char *msg = pcc_last_error();
    if (rc != want) {
        fprintf(stderr, "%s: returned %d, expected %d (%s)\n", call, rc, want, msg ? msg : "");
        ++failures;
        return;
    }
    if (want != PCC_OK && (!msg || !strstr(msg, call))) {
        fprintf(stderr, "%s: message does not name the call: '%s'\n", call, msg ? msg : "(null)");
        ++failures;
    }
}

int main(void)
{
    const char *v = pcc_version();
    if (!v || strncmp(v, "pcc", 3) != 0) {
        fprintf(stderr, "pcc_version: '%s'\n", v ? v : "(null)");
        ++failures;
    }

    /* return-code and status-bit names */
    if (strncmp(pcc_status_string(PCC_E_CAPACITY), "PCC_E_CAPACITY", 14) != 0 ||
        strcmp(pcc_status_string(99), "unknown return code") != 0 ||
        strcmp(pcc_status_bit_string(PCC_ST_TIMEOUT), "PCC_ST_TIMEOUT") != 0 ||
        strcmp(pcc_status_bit_string(PCC_ST_TIMEOUT | PCC_ST_CAPACITY), "unknown status bit") != 0) {
        fprintf(stderr, "status strings\n");
        ++failures;
    }

    pcc_ctx *ctx = (pcc_ctx *)&failures;   /* must be overwritten with NULL */
    expect(pcc_create(NULL, 0), PCC_E_INVALID, "pcc_create");
    int rc = pcc_create(&ctx, -1);
    if (rc == PCC_OK || ctx != NULL) {
        fprintf(stderr, "pcc_create(-1): rc %d, ctx %p\n", rc, (void *)ctx);
        ++failures;
        if (rc == PCC_OK) pcc_destroy(ctx);
    }
    pcc_destroy(NULL);

    pcc_material mat;
    memset(&mat, 0, sizeof mat);
    pcc_table_spec spec;
    memset(&spec, 0, sizeof spec);
    pcc_species sp;
    memset(&sp, 0, sizeof sp);
    pcc_particles parts;
    memset(&parts, 0, sizeof parts);
    pcc_cells cells;
    memset(&cells, 0, sizeof cells);
    pcc_step_desc desc;
    memset(&desc, 0, sizeof desc);
    pcc_stats stats;
    unsigned status = 0;
    double d[8];
    float f[8];
    int iv[8];
    uint32_t u[8];
    float ms = 0.0f;

    /* every call that takes a context rejects a null one */
    expect(pcc_tables_build(NULL, &mat, 1, &spec, NULL), PCC_E_INVALID, "pcc_tables_build");
    expect(pcc_tables_read(NULL, d, d, d, d, d, d, d), PCC_E_INVALID, "pcc_tables_read");
    expect(pcc_bin(NULL, &parts, 1, &sp, 0, 1.0, NULL), PCC_E_INVALID, "pcc_bin");
    expect(pcc_collide(NULL, &cells, &sp, &sp, &sp, &sp, 1e-15, 1, 0, 7u, 0, NULL, NULL), PCC_E_INVALID,
           "pcc_collide");
    expect(pcc_set_schedule(NULL, 1, 1), PCC_E_INVALID, "pcc_set_schedule");
    expect(pcc_set_wait_limit(NULL, 1), PCC_E_INVALID, "pcc_set_wait_limit");
    {
        int thr[4] = {20, 18, 14, 0};
        expect(pcc_set_scan_classes(NULL, 0, thr), PCC_E_INVALID, "pcc_set_scan_classes");
        expect(pcc_get_scan_classes(NULL, 0, thr), PCC_E_INVALID, "pcc_get_scan_classes");
    }
    expect(pcc_append_secondaries(NULL, 1, &sp, NULL), PCC_E_INVALID, "pcc_append_secondaries");
    expect(pcc_pairing(NULL, 1, &sp, &sp, 0, 1, 0, iv, iv, NULL), PCC_E_INVALID, "pcc_pairing");
    expect(pcc_totals(NULL, 1, &sp, 0, d, NULL), PCC_E_INVALID, "pcc_totals");
    expect(pcc_steps_capture(NULL, &desc, 0, 1, 0, NULL), PCC_E_INVALID, "pcc_steps_capture");
    expect(pcc_steps_launch(NULL, NULL), PCC_E_INVALID, "pcc_steps_launch");
    expect(pcc_steps_timing(NULL, &ms), PCC_E_INVALID, "pcc_steps_timing");
    expect(pcc_read_status(NULL, &status, &stats, NULL), PCC_E_INVALID, "pcc_read_status");
    expect(pcc_expected_emission_fwd(NULL, 1, 1, 29, 8, f, f, f, f, NULL), PCC_E_INVALID,
           "pcc_expected_emission_fwd");
    expect(pcc_expected_emission_bwd(NULL, 1, 1, 29, 8, f, f, f, f, f, NULL), PCC_E_INVALID,
           "pcc_expected_emission_bwd");

    /* the context-free calls check their arrays and sizes first */
    expect(pcc_accept_check(-1, u, d, u, u, u, 0, 0, iv, iv, NULL), PCC_E_INVALID, "pcc_accept_check");
    expect(pcc_accept_check(4, NULL, d, u, u, u, 0, 0, iv, iv, NULL), PCC_E_INVALID, "pcc_accept_check");
    expect(pcc_accept_check(4, u, d, u, u, u, 0, 0, iv, NULL, NULL), PCC_E_INVALID, "pcc_accept_check");
    expect(pcc_accept_check(0, NULL, NULL, NULL, NULL, NULL, 0, 0, NULL, NULL, NULL), PCC_OK,
           "pcc_accept_check");
    expect(pcc_totals_noalloc(1, NULL, 0, d, NULL), PCC_E_INVALID, "pcc_totals_noalloc");
    expect(pcc_totals_noalloc(1, &sp, 0, d, NULL), PCC_E_INVALID, "pcc_totals_noalloc");
    /* a fully populated descriptor (host addresses, never dereferenced)
     * with too many cells for the fixed scratch: PCC_E_CAPACITY */
    sp.ux = sp.uy = sp.uz = sp.w = f;
    sp.cell_start = sp.cell_count = iv;
    expect(pcc_totals_noalloc(0, &sp, 0, d, NULL), PCC_E_INVALID, "pcc_totals_noalloc");
    expect(pcc_totals_noalloc(1 << 30, &sp, 0, d, NULL), PCC_E_CAPACITY, "pcc_totals_noalloc");

    if (pcc_launch_count() != 0) {
        fprintf(stderr, "rejected calls launched %llu kernels\n", pcc_launch_count());
        ++failures;
    }
    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("C ABI sanitizer driver: all checks passed\n");
    return 0;
}
