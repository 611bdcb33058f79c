/* A plain C client of the library: the stream interface only (include/rfsr.h, librfsr.so).
 * Reads F frames of H x W samples and masks from a binary file (samples then mask per frame),
 * reconstructs them through rfsr_push_frame / rfsr_get_frame with two frames in flight, and
 * writes the 8-bit reconstructions to a second file.
 *   usage: rfsr_c_client H W F input.bin output.bin */
#include <stdio.h>
#include <stdlib.h>

#include "rfsr.h"

static int check(int rc, const char *what)
{
    if (rc < 0) fprintf(stderr, "%s failed: %d (%s)\n", what, rc, rfsr_last_error());
    return rc < 0;
}

int main(int argc, char **argv)
{
    if (argc != 6) {
        fprintf(stderr, "usage: %s H W F input.bin output.bin\n", argv[0]);
        return 2;
    }
    const int H = atoi(argv[1]), W = atoi(argv[2]), F = atoi(argv[3]);
    const size_t HW = (size_t)H * W;
    unsigned char *in = malloc(2 * HW * F), *out = malloc(HW * F);
    FILE *fi = fopen(argv[4], "rb");
    if (!in || !out || !fi || fread(in, 1, 2 * HW * F, fi) != 2 * HW * F) return 2;
    fclose(fi);

    rfsr_engine_config ec;
    rfsr_engine_config_default(&ec);
    rfsr_engine *eng = NULL;
    if (check(rfsr_engine_create(&ec, &eng), "rfsr_engine_create")) return 1;
    rfsr_stream_config sc;
    rfsr_stream_config_default(&sc);
    sc.height = H;
    sc.width = W;
    rfsr_stream *st = NULL;
    if (check(rfsr_create_stream(eng, &sc, &st), "rfsr_create_stream")) return 1;
    int pushed = 0;
    for (int t = 0; t < F; ++t) {
        while (pushed < F && pushed <= t + 1) {            /* keep two frames in flight */
            const unsigned char *f = in + 2 * HW * pushed;
            if (check(rfsr_push_frame(st, f, f + HW), "rfsr_push_frame")) return 1;
            ++pushed;
        }
        if (check(rfsr_get_frame(st, out + HW * t, NULL, 60000), "rfsr_get_frame")) return 1;
    }
    if (check(rfsr_destroy(st), "rfsr_destroy")) return 1;
    if (check(rfsr_engine_destroy(eng), "rfsr_engine_destroy")) return 1;
    FILE *fo = fopen(argv[5], "wb");
    if (!fo || fwrite(out, 1, HW * F, fo) != HW * F) return 2;
    fclose(fo);
    free(in);
    free(out);
    return 0;
}
