// compress_static.cu -- szx_compress_static_async: compression whose scratch
// is a fixed array inside this library instead of the tail of the caller's
// output buffer.
//
// Why it exists: szx_compress_async needs the caller's buffer to be larger
// than the stream (szx_compress_bound = stream maximum + look-back
// workspace).  Some callers cannot provide those extra bytes and cannot
// allocate them either: a caller writing each stream into a slot of a
// pre-partitioned arena sized exactly to szx_stream_max_bytes, or one running
// a latency-bound loop where a cudaMalloc (which may synchronise the device)
// or a pool allocation is not allowed.  This entry point serves them: it
// allocates nothing at all, on the device or through any library.
//
// The look-back workspace (a 128-byte header of counters plus one 8-byte
// flag word per tile) lives in g_static_ws below.  Its device address is
// looked up once per device with cudaGetSymbolAddress, under a mutex, on the
// first call made with that device current; later calls reuse it.  So a
// cudaDeviceReset between calls (which reloads the module, possibly at
// another address) is not supported, as szx.h states.  Every
// call clears the part of the array it uses (a clear kernel on the caller's
// stream) before the kernel starts, because the tile counters and look-back
// flags must start at zero.  All calls on one device share the array, so two
// calls that can overlap in time (different streams, or different host
// threads) race on it; callers must order them.
#include "szx.h"
#include "szx_device.cuh"
#include "szx_host.h"
#include "szx_launch.h"

#include <cmath>
#include <cstring>
#include <mutex>

using namespace szx;

namespace {

static_assert(SZX_STATIC_SCRATCH_BYTES % 256 == 0, "scratch size is a multiple of 256");
static_assert(SZX_STATIC_MAX_TILES == (SZX_STATIC_SCRATCH_BYTES - kWsHeader) / 8,
              "tile limit matches the scratch size");

static __device__ __align__(256) unsigned char g_static_ws[SZX_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ws_ptr[kMaxDevices] = {};

// Address of g_static_ws on the current device (looked up once per device).
szx_status static_ws(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SZX_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ws_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return SZX_ERR_CUDA;
        g_ws_ptr[dev] = p;
    }
    *out = g_ws_ptr[dev];
    return SZX_OK;
}

}  // namespace

extern "C" szx_status szx_compress_static_async(const void *d_in, size_t n, szx_dtype dtype, double eb,
                                                uint32_t block, void *d_out, size_t out_capacity,
                                                uint64_t *d_result, szx_stream_t stream) {
    if (!d_in || !d_out || (dtype != SZX_F32 && dtype != SZX_F64) || !block_ok(block)) return SZX_ERR_INVALID;
    if (!(eb > 0.0) || !std::isfinite(eb)) return SZX_ERR_INVALID;
    if (!aligned16(d_in) || !aligned16(d_out)) return SZX_ERR_INVALID;
    const size_t smax = szx_stream_max_bytes(n, dtype, block);
    if (!smax) return SZX_ERR_INVALID;  // n == 0 or n above the library's limit
    const uint32_t w = dtype == SZX_F32 ? 4u : 8u;
    const Geometry g = make_geometry(n, block, w);
    if (g.ntiles > SZX_STATIC_MAX_TILES) return SZX_ERR_INVALID;  // beyond the fixed scratch
    if (out_capacity < smax) return SZX_ERR_TOO_SMALL;
    void *ws = nullptr;
    const szx_status st = static_ws(&ws);
    if (st != SZX_OK) return st;
    const cudaError_t e = launch_compress_ws(d_in, n, (int)dtype, bound_bits(eb, dtype), block, d_out, ws,
                                             d_result, (cudaStream_t)stream);
    return e == cudaSuccess ? SZX_OK : SZX_ERR_CUDA;
}
