/*
 * A plain C client of the library: no Python, no PyTorch, no CUDA headers.
 * It reads a mesh and a batch of segments from a binary file, builds the
 * hierarchy from host memory (lbvh_build_host), answers the boolean and the
 * intercept_count queries of Sec. 1 from host memory (rsi_query_host) and
 * writes the answers to a second file.  The tests compare them with the
 * oracle.
 *
 * Input : int64 n_vertices, n_triangles, n_rays; float vertices[n_v][3];
 *         int32 triangles[n_t][3]; float from[n_r][3]; float to[n_r][3].
 * Output: uint8 hit[n_r]; uint8 ambiguous (boolean)[n_r];
 *         int32 count[n_r]; uint8 ambiguous (count)[n_r].
 * Exit status 0 on success; otherwise the library's message on stderr.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "rsi.h"

static int read_all(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

int main(int argc, char** argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s input output\n", argv[0]);
        return 2;
    }
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 2;
    int64_t nv = 0, nt = 0, nr = 0;
    if (!read_all(in, &nv, 8) || !read_all(in, &nt, 8) || !read_all(in, &nr, 8) || nv < 1 || nt < 1 || nr < 0)
        return 2;
    float* V = malloc(12 * (size_t)nv);
    int32_t* T = malloc(12 * (size_t)nt);
    float* F = malloc(12 * (size_t)nr + 1);
    float* E = malloc(12 * (size_t)nr + 1);
    uint8_t* hit = malloc((size_t)nr + 1);
    uint8_t* amb_hit = malloc((size_t)nr + 1);
    int32_t* count = malloc(4 * (size_t)nr + 1);
    uint8_t* amb_count = malloc((size_t)nr + 1);
    if (!V || !T || !F || !E || !hit || !amb_hit || !count || !amb_count) return 2;
    if (!read_all(in, V, 12 * (size_t)nv) || !read_all(in, T, 12 * (size_t)nt) || !read_all(in, F, 12 * (size_t)nr) ||
        !read_all(in, E, 12 * (size_t)nr))
        return 2;
    fclose(in);

    rsi_bvh_t h = NULL;
    if (lbvh_build_host(V, nv, T, nt, (int)sizeof(int32_t), 30, NULL, &h) != RSI_OK) {
        fprintf(stderr, "lbvh_build_host: %s\n", rsi_last_error());
        return 1;
    }
    rsi_bvh_info info;
    rsi_stats st;
    if (lbvh_info(h, &info) != RSI_OK ||
        rsi_query_host(h, F, E, nr, RSI_ANY_HIT, NULL, hit, NULL, amb_hit, NULL, NULL) != RSI_OK ||
        rsi_query_host(h, F, E, nr, RSI_COUNT, NULL, NULL, count, amb_count, &st, NULL) != RSI_OK) {
        fprintf(stderr, "query: %s\n", rsi_last_error());
        lbvh_free(h);
        return 1;
    }
    lbvh_free(h);

    FILE* out = fopen(argv[2], "wb");
    if (!out) return 2;
    fwrite(hit, 1, (size_t)nr, out);
    fwrite(amb_hit, 1, (size_t)nr, out);
    fwrite(count, 4, (size_t)nr, out);
    fwrite(amb_count, 1, (size_t)nr, out);
    fclose(out);
    printf("triangles %lld, tree height %d, segments %lld, queued for FP64 %lld, ambiguous %lld\n",
           (long long)info.n_triangles, info.height, (long long)nr, (long long)st.band_rays,
           (long long)st.ambiguous);
    free(V), free(T), free(F), free(E), free(hit), free(amb_hit), free(count), free(amb_count);
    return 0;
}
