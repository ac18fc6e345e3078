/* Test driver: runs the oracle on an event read from a file, for the sanitizer test
 * (tests/test_oracle_sanitizers.py builds it with -fsanitize=address,undefined).
 * File layout (native endianness): int64 n, int32 n_rows, int32 n_sectors, double row_x[n_rows],
 * double y[n], double z[n], uint8 row[n], int32 counts[n_sectors * n_rows]. */
#include <stdio.h>
#include <stdlib.h>
#include "oracle.h"

static void *read_n(FILE *f, size_t bytes)
{
    void *p = malloc(bytes > 0 ? bytes : 1);
    if (bytes && fread(p, 1, bytes, f) != bytes) {
        fprintf(stderr, "short read\n");
        exit(2);
    }
    return p;
}

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t n;
    int32_t nr, ns;
    if (fread(&n, 8, 1, f) != 1 || fread(&nr, 4, 1, f) != 1 || fread(&ns, 4, 1, f) != 1) return 2;
    double *rx = read_n(f, sizeof(double) * (size_t)nr);
    double *y = read_n(f, sizeof(double) * (size_t)n);
    double *z = read_n(f, sizeof(double) * (size_t)n);
    uint8_t *row = read_n(f, (size_t)n);
    int32_t *counts = read_n(f, sizeof(int32_t) * (size_t)nr * (size_t)ns);
    fclose(f);
    for (int flags = 0; flags < 4; flags++) {
        orc_config c;
        orc_default_config(&c, rx, nr, ns);
        c.n_threads = 1;
        c.global_tracking = flags & 1;
        c.merge = (flags >> 1) & 1;
        for (int prec = 0; prec < 2; prec++) {
            orc_result *r = prec ? orc_track_event_f64(&c, y, z, row, counts, n) : orc_track_event_f32(&c, y, z, row, counts, n);
            int64_t info[ORC_INFO_COUNT];
            void *ptrs[ORC_PTR_COUNT];
            orc_result_info(r, info);
            orc_result_ptrs(r, ptrs);
            printf("flags %d precision %d tracks %lld merged %lld\n", flags, prec ? 64 : 32,
                   (long long)info[ORC_INFO_N_TRACKS], (long long)info[ORC_INFO_N_MERGED]);
            orc_result_free(r);
        }
    }
    free(rx);
    free(y);
    free(z);
    free(row);
    free(counts);
    return 0;
}
