// szx_launch.h -- internal launchers behind the C ABI (not part of the ABI).
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cuda_runtime.h>

#include "szx.h"

namespace szx {

// How a single-field launch zeroes its scratch or status words first:
//   kernel    -- a clear kernel (launch_clear_words), with the codec kernel as
//                its programmatic dependent: the shorter on the GPU, for
//                calls back to back on one stream;
//   memset    -- a cudaMemsetAsync and a plain launch: about 1.7 us less host
//                time per call, and the faster when many streams run such
//                calls at once (the serving loop's slots), where a small
//                kernel has to wait for room on an SM;
//   automatic -- kernel for launches of at least kClearKernelMinTiles tiles,
//                memset below, where a call back to back with others is
//                bound by the host's launch time rather than the GPU.
enum class Clear { kernel, memset, automatic };
constexpr uint64_t kClearKernelMinTiles = 256;

// szx_compress_async and szx_decompress_async with the clear mode chosen (the
// public calls use Clear::automatic; the serving loop, Clear::memset).
szx_status compress_async_with(const void *d_in, size_t n, szx_dtype dtype, double eb, uint32_t block, void *d_out,
                               size_t out_capacity, uint64_t *d_result, szx_stream_t stream, Clear clear);
szx_status decompress_async_with(const void *d_in, size_t in_bytes, const szx_header *h, void *d_out,
                                 size_t out_capacity, uint32_t *d_status, szx_stream_t stream, Clear clear);

// Zero n 4-byte words at p (device memory) on `stream`, with a small kernel
// (not a memset node) so that the kernel enqueued right after it can be
// launched as its programmatic dependent (launch_kernel with pdl).
cudaError_t launch_clear_words(uint32_t *p, uint64_t n, cudaStream_t stream);

// kern<<<grid, threads, smem, stream>>>(args...).  With pdl, as the
// programmatic dependent of the kernel before it on the stream: its CTAs may
// start, and run what precedes their wait_prior_grids(), while that kernel
// still runs.  Only kernels that call wait_prior_grids() before their first
// global-memory access may be launched so.
template <typename... P, typename... A>
cudaError_t launch_kernel(void (*kern)(P...), unsigned grid, unsigned threads, size_t smem, bool pdl,
                          cudaStream_t stream, A &&...args) {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1u : 0u;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<A &&>(args)...);
}

// Limit (microseconds) of a bounded device-side wait: the environment variable
// `name` (a positive integer) if set, else `fallback`.  Read on every launch.
uint32_t wait_limit_from_env(const char *name, uint32_t fallback);

// Per (device, kernel, shared-memory size), on first use: raise the kernel's
// dynamic shared-memory limit to smem and look up how many CTAs of `threads`
// threads fit on an SM and how many SMs the device has; later calls return the
// cached values (a hash map under a mutex).
cudaError_t launch_setup(const void *kernel, uint32_t smem, int threads, int *per_sm, int *sms);

// Encode a 2-D TMA tensor map over `rows` rows of 128 bytes at base (32-bit
// elements, a box of 32 x box_rows (<= 256), 128-byte swizzle).  False if
// rows is 0 or >= 2^31, or the driver entry point is unavailable or rejects
// the map.
bool encode_row_map(CUtensorMap *tm, const void *base, uint64_t rows, uint32_t box_rows);

// Enqueue the compression of n values (dtype 0 = f32, 1 = f64) with bound bits
// e_bits into the stream at out; the workspace starts ws_offset bytes into
// out.  Optionally writes {stream bytes, status} to d_result on completion.
cudaError_t launch_compress(const void *in, uint64_t n, int dtype, uint64_t e_bits, uint32_t block,
                            void *out, uint64_t ws_offset, uint64_t *d_result, cudaStream_t stream,
                            Clear clear = Clear::automatic);

// Same, with the workspace (workspace_bytes(ntiles) bytes, 256-byte aligned)
// at an arbitrary device address instead of the tail of out.  Clears it on
// `stream` first, as `clear` says.
cudaError_t launch_compress_ws(const void *in, uint64_t n, int dtype, uint64_t e_bits, uint32_t block,
                               void *out, void *ws, uint64_t *d_result, cudaStream_t stream,
                               Clear clear = Clear::automatic);

struct CField;

// Fill the descriptor of one field for a batched compression launch (host
// memory; the tensor map is encoded here).  ws: the field's workspace
// (workspace_bytes(ntiles), zeroed before the launch); tile0: the field's first
// tile in the launch's global list.
void fill_compress_field(CField *f, const void *in, uint64_t n, int dtype, uint64_t e_bits, uint32_t block,
                         void *out, void *ws, uint64_t *d_result, uint64_t tile0);

// Enqueue one persistent compression launch over the nfields descriptors at
// d_fields (device memory, 64-byte aligned; all of dtype and block), whose
// tiles number total_tiles.  d_counters: 3 zeroed words (ticket, done, error
// bits).  ctas_per_sm: 0 = as many as fit, else at most that many.  nw: the
// consumer warps per CTA, 8 or 4 (0 = 8; see kernel_shape_ok).  pdl: launch
// as the programmatic dependent of the kernel before it (launch_kernel).
cudaError_t launch_compress_batch(const void *d_fields, uint32_t nfields, uint64_t total_tiles, uint32_t *d_counters,
                                  int dtype, uint32_t block, int ctas_per_sm, int nw, bool pdl, cudaStream_t stream);

// Whether the kernels have an instance with nw consumer (decoding) warps for
// this dtype and block: 8 always; 4 where a block covers whole lanes of 64
// values (f32, b >= 64) or 32 values (f64, b <= 512).
inline bool kernel_shape_ok(int dtype, uint32_t block, int nw) {
    if (nw == 8) return true;
    if (nw != 4) return false;
    return dtype == 0 ? block >= 64 : block <= 512;
}

struct DField;

// Fill the descriptor of one stream for a batched decompression launch (host
// memory; the output tensor map is encoded here).
// blk_lo, blk_hi: the blocks written (out holds values from block blk_lo on);
// 0 and UINT64_MAX for the whole stream.
void fill_decompress_field(DField *f, const void *in, uint64_t total_bytes, uint64_t n, int dtype, uint32_t block,
                           void *out, uint32_t *d_status, bool check_header, uint64_t tile0, uint64_t blk_lo = 0,
                           uint64_t blk_hi = ~0ull);

// Tiles a filled descriptor decodes.
uint64_t decompress_field_tiles(const DField *f);

// Enqueue one persistent decompression launch over nfields descriptors at
// d_fields (device memory, 64-byte aligned; all of dtype and block).  CTAs
// take tiles by ticket from *d_ticket (device memory, zero before the launch),
// or, if d_ticket is null, by a static split.
cudaError_t launch_decompress_batch(const void *d_fields, uint32_t nfields, uint64_t total_tiles, uint32_t *d_ticket,
                                    int dtype, uint32_t block, int ctas_per_sm, int nw, bool pdl,
                                    cudaStream_t stream);

// Enqueue the decompression of a stream of total_bytes whose header says
// (n, dtype, block).  *d_status is zeroed on `stream` first, as `clear` says,
// and errors are folded into it with atomicMax as szx_status codes (d_status
// may be null).
cudaError_t launch_decompress(const void *in, uint64_t in_bytes, uint64_t total_bytes, uint64_t n, int dtype,
                              uint32_t block, void *out, uint32_t *d_status, bool check_header,
                              cudaStream_t stream, uint64_t blk_lo = 0, uint64_t blk_hi = ~0ull,
                              Clear clear = Clear::automatic);

}  // namespace szx
