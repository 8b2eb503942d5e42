/*
 * szx_ref.h -- the CPU oracle of the SZx block codec.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke() check of
 * __graft_entry__.py and the cpu_baseline / reference arm of bench.py may
 * build, load or call anything under oracle/.  The CUDA library never links
 * it, and the two share no source, header, table or helper.
 *
 * It is a plain, single-threaded restatement of Algorithm 1 of the paper
 * (Sec. IV), Eq. 4 (required bits), Eq. 5 (byte-alignment right shift) and
 * the lead-code / mid-byte description that follows Algorithm 1, plus the
 * exact inverse (decompression, Sec. V-B).  It fixes the byte layout of the
 * compressed stream, which the paper leaves open; the layout and every
 * reading of the paper it relies on are stated in szx_ref.c.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 *        szx_ref.c -o liboracle.so -lm      (oracle/build.py does this)
 */
#ifndef SZX_REF_H
#define SZX_REF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* dtype codes */
#define SZX_REF_F32 0
#define SZX_REF_F64 1

/* status codes (same meanings as the library's, declared independently) */
#define SZX_REF_OK 0
#define SZX_REF_ERR_INVALID 1
#define SZX_REF_ERR_TOO_SMALL 2
#define SZX_REF_ERR_CORRUPT 3

/* Worst-case stream size for n values of dtype with block length `block`. */
size_t szx_ref_compress_bound(size_t n, int dtype, uint32_t block);

/*
 * Compress n values (host memory, little-endian IEEE 754) with absolute
 * error bound eb.  Writes the stream to out[0 .. *out_bytes).  Returns a
 * status code; on error nothing useful is in out.
 */
int szx_ref_compress(const void *in, size_t n, int dtype, double eb,
                     uint32_t block, void *out, size_t cap, size_t *out_bytes);

/*
 * Decompress a stream.  *n_out and *dtype_out receive the header's values;
 * out must hold n * (4 or 8) bytes.  Returns SZX_REF_ERR_CORRUPT for any
 * malformed stream (no read outside in[0 .. in_bytes)).
 */
int szx_ref_decompress(const void *in, size_t in_bytes, void *out, size_t cap,
                       size_t *n_out, int *dtype_out);

/* The absolute bound actually used for dtype: f32 rounds eb toward zero. */
uint64_t szx_ref_error_bound_bits(double eb, int dtype);

/*
 * Diagnostics of Sec. V-A.1 (Eq. 6): over the non-constant, non-raw blocks,
 * bits_c = sum over values of (reqBits + s - 8 L_i), the bits stored with the
 * right shift, and bits_ab = sum over values of (reqBits - 8 L0_i), the bits an
 * unshifted, bit-granular packing (Solutions A/B) stores, where L0_i counts
 * identical leading bytes of the unshifted truncated words.  Returns a status.
 */
int szx_ref_shift_overhead_bits(const void *in, size_t n, int dtype, double eb,
                                uint32_t block, uint64_t *bits_c,
                                uint64_t *bits_ab);

#ifdef __cplusplus
}
#endif
#endif /* SZX_REF_H */
