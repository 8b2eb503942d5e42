/*
 * A plain C user of the library's ABI (include/szx.h): no Python in the calls.
 * Compresses n f32 values with szx_compress, decompresses them with
 * szx_decompress, decodes a block range with szx_decompress_range_async, and
 * writes the input, the stream, the decoded values and the range to files
 * for the test to compare with the oracle.  Usage: c_program DIR
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "szx.h"

static int write_file(const char *dir, const char *name, const void *p, size_t bytes) {
    char path[4096];
    snprintf(path, sizeof(path), "%s/%s", dir, name);
    FILE *f = fopen(path, "wb");
    if (!f) return 1;
    size_t w = fwrite(p, 1, bytes, f);
    fclose(f);
    return w != bytes;
}

#define CHECK_CUDA(x)                                                             \
    do {                                                                          \
        cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) {                                                  \
            fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));              \
            return 2;                                                             \
        }                                                                         \
    } while (0)

int main(int argc, char **argv) {
    if (argc < 2) return 64;
    const size_t n = (1u << 20) + 321;
    const uint32_t block = 128;
    float *x = (float *)malloc(n * sizeof(float));
    float *y = (float *)malloc(n * sizeof(float));
    uint64_t s = 88172645463325252ull;  /* xorshift64 */
    for (size_t i = 0; i < n; ++i) {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        const double noise = ((double)(s >> 11) / 9007199254740992.0 - 0.5) * 0.02;
        x[i] = (float)(sin(i * 0.001) + 0.5 * sin(i * 0.0173) + noise);
    }
    const double eb = 1e-3;
    void *d_x, *d_y, *d_out, *d_part;
    const size_t cap = szx_compress_bound(n, SZX_F32, block);
    CHECK_CUDA(cudaMalloc(&d_x, n * sizeof(float)));
    CHECK_CUDA(cudaMalloc(&d_y, n * sizeof(float)));
    CHECK_CUDA(cudaMalloc(&d_out, cap));
    CHECK_CUDA(cudaMemcpy(d_x, x, n * sizeof(float), cudaMemcpyHostToDevice));

    size_t nbytes = 0;
    szx_status st = szx_compress(d_x, n, SZX_F32, eb, block, d_out, cap, &nbytes, 0);
    if (st != SZX_OK) {
        fprintf(stderr, "szx_compress: %s\n", szx_status_string(st));
        return 3;
    }
    size_t n_out = 0;
    szx_dtype dt;
    st = szx_decompress(d_out, nbytes, d_y, n * sizeof(float), &n_out, &dt, 0);
    if (st != SZX_OK || n_out != n || dt != SZX_F32) {
        fprintf(stderr, "szx_decompress: %s\n", szx_status_string(st));
        return 4;
    }
    /* blocks 100..299 alone */
    szx_header h;
    st = szx_header_read(d_out, nbytes, &h, 0);
    if (st != SZX_OK) return 5;
    const size_t first = 100, count = 200;
    CHECK_CUDA(cudaMalloc(&d_part, count * block * sizeof(float)));
    st = szx_decompress_range_async(d_out, nbytes, &h, first, count, d_part, count * block * sizeof(float),
                                    NULL, 0);
    if (st != SZX_OK) return 6;
    CHECK_CUDA(cudaDeviceSynchronize());

    uint8_t *stream = (uint8_t *)malloc(nbytes);
    float *part = (float *)malloc(count * block * sizeof(float));
    CHECK_CUDA(cudaMemcpy(stream, d_out, nbytes, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(y, d_y, n * sizeof(float), cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(part, d_part, count * block * sizeof(float), cudaMemcpyDeviceToHost));
    if (write_file(argv[1], "x.bin", x, n * sizeof(float)) || write_file(argv[1], "stream.bin", stream, nbytes) ||
        write_file(argv[1], "y.bin", y, n * sizeof(float)) ||
        write_file(argv[1], "part.bin", part, count * block * sizeof(float)))
        return 7;
    printf("ok %zu values -> %zu bytes (%s)\n", n, nbytes, szx_version());
    cudaFree(d_x);
    cudaFree(d_y);
    cudaFree(d_out);
    cudaFree(d_part);
    free(x);
    free(y);
    free(stream);
    free(part);
    return 0;
}
