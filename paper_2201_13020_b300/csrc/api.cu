// api.cu -- the extern "C" surface declared in include/szx.h.
//
// Host-side argument checks, the stream geometry, and the launch sequence on
// the caller's stream.  Every device step is one of this library's kernels
// (the scratch and status words are cleared by one too); there is no host or
// CPU fallback: if the kernels cannot run, the call returns SZX_ERR_CUDA.
#include "szx.h"
#include "szx_device.cuh"
#include "szx_host.h"
#include "szx_launch.h"

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>

using namespace szx;

namespace {

constexpr uint64_t kMaxValues = 1ull << 40;

bool dtype_ok(szx_dtype d) { return d == SZX_F32 || d == SZX_F64; }
uint32_t width(szx_dtype d) { return d == SZX_F32 ? 4u : 8u; }
uint64_t align256(uint64_t x) { return align_up(x, 256); }

uint64_t stream_max(uint64_t n, uint32_t b, uint32_t w) {
    const Geometry g = make_geometry(n, b, w);
    const uint64_t full = g.ntiles - 1;
    const uint64_t last_blocks = g.nb - full * g.G;
    const uint64_t last_vals = n - full * g.G * b;
    return g.off_rec + full * record_max_bytes(g.G, b, w) +
           pad16(last_blocks * (b / 4 + 1) + last_vals * w);
}

szx_status from_cuda(cudaError_t e) { return e == cudaSuccess ? SZX_OK : SZX_ERR_CUDA; }

// Status words of the synchronous decompress: a fixed array in the library's
// device memory (every device that loads the library holds one), so the call
// allocates nothing.  Its address is looked up on every call (a host-side
// lookup once the module is loaded).  Calls take words round-robin, so up to
// kSlots calls in flight at once get distinct words.
constexpr int kSlots = 256;
static __device__ __align__(256) uint32_t g_sync_status[kSlots];
std::atomic<uint32_t> g_slot{0};

uint32_t *status_slot(szx_status *st) {
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_sync_status) != cudaSuccess || !base) {
        *st = SZX_ERR_CUDA;
        return nullptr;
    }
    *st = SZX_OK;
    return static_cast<uint32_t *>(base) + (g_slot.fetch_add(1) % kSlots);
}

szx_status parse_header(const uint8_t *h, uint64_t in_bytes, szx_header *out) {
    uint32_t h32[4];
    uint64_t h64[8];
    std::memcpy(h32, h, 16);
    std::memcpy(h64, h, 64);
    if (h32[0] != kMagic || (h32[1] & 0xFFu) != kVersion || (h32[1] >> 16) != 0) return SZX_ERR_CORRUPT;
    const uint32_t dt = (h32[1] >> 8) & 0xFFu;
    if (dt > 1) return SZX_ERR_CORRUPT;
    const szx_dtype d = (szx_dtype)dt;
    const uint32_t b = h32[2];
    if (!block_ok(b) || h32[3] != tile_blocks(b, width(d))) return SZX_ERR_CORRUPT;
    const uint64_t n = h64[2];
    if (n == 0 || n > kMaxValues) return SZX_ERR_CORRUPT;
    const Geometry g = make_geometry(n, b, width(d));
    const uint64_t total = h64[7];
    if (total > in_bytes || total < g.off_rec || (total & 15)) return SZX_ERR_CORRUPT;
    out->block = b;
    out->tile_blocks = h32[3];
    out->n = n;
    out->dtype = d;
    out->e_bits = h64[3];
    out->nonconst = h64[4];
    out->raw = h64[5];
    out->escalated = h64[6];
    out->total_bytes = total;
    return SZX_OK;
}

szx_status check_compress_args(const void *d_in, size_t n, szx_dtype dtype, double eb, uint32_t block,
                               const void *d_out, size_t out_capacity) {
    if (!d_in || !d_out || !dtype_ok(dtype) || !block_ok(block)) return SZX_ERR_INVALID;
    if (n == 0 || n > kMaxValues) return SZX_ERR_INVALID;
    if (!(eb > 0.0) || !std::isfinite(eb)) return SZX_ERR_INVALID;
    if (!aligned16(d_in) || !aligned16(d_out)) return SZX_ERR_INVALID;
    if (out_capacity < szx_compress_bound(n, dtype, block)) return SZX_ERR_TOO_SMALL;
    return SZX_OK;
}

}  // namespace

namespace {
struct SetupKey {
    int dev;
    const void *kernel;
    uint32_t smem;
    bool operator==(const SetupKey &o) const { return dev == o.dev && kernel == o.kernel && smem == o.smem; }
};
struct SetupHash {
    size_t operator()(const SetupKey &k) const {
        return std::hash<const void *>()(k.kernel) ^ (size_t)k.dev * 0x9E3779B97F4A7C15ull ^ (size_t)k.smem << 17;
    }
};
std::mutex g_setup_mu;
std::unordered_map<SetupKey, std::pair<int, int>, SetupHash> g_setup;
}  // namespace

cudaError_t szx::launch_setup(const void *kernel, uint32_t smem, int threads, int *per_sm, int *sms) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const SetupKey key{dev, kernel, smem};
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        auto it = g_setup.find(key);
        if (it != g_setup.end()) {
            *per_sm = it->second.first;
            *sms = it->second.second;
            return cudaSuccess;
        }
    }
    if ((err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return err;
    int n_sm = 0, fit = 0;
    if ((err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, threads, smem)) != cudaSuccess) return err;
    if (fit < 1) return cudaErrorInvalidConfiguration;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    g_setup[key] = {fit, n_sm};
    *per_sm = fit;
    *sms = n_sm;
    return cudaSuccess;
}

uint32_t szx::wait_limit_from_env(const char *name, uint32_t fallback) {
    const char *v = std::getenv(name);
    if (!v || !*v) return fallback;
    char *end = nullptr;
    const unsigned long long x = std::strtoull(v, &end, 10);
    if (end == v || x == 0 || x > 0xFFFFFFFFull) return fallback;
    return (uint32_t)x;
}

namespace szx {

szx_status compress_async_with(const void *d_in, size_t n, szx_dtype dtype, double eb, uint32_t block, void *d_out,
                               size_t out_capacity, uint64_t *d_result, szx_stream_t stream, Clear clear) {
    szx_status st = check_compress_args(d_in, n, dtype, eb, block, d_out, out_capacity);
    if (st != SZX_OK) return st;
    const uint64_t ws = align256(stream_max(n, block, width(dtype)));
    return from_cuda(launch_compress(d_in, n, (int)dtype, bound_bits(eb, dtype), block, d_out, ws, d_result,
                                     (cudaStream_t)stream, clear));
}

szx_status decompress_async_with(const void *d_in, size_t in_bytes, const szx_header *h, void *d_out,
                                 size_t out_capacity, uint32_t *d_status, szx_stream_t stream, Clear clear) {
    if (!d_in || !h || !d_out) return SZX_ERR_INVALID;
    if (!aligned16(d_in) || !aligned16(d_out)) return SZX_ERR_INVALID;
    if (!dtype_ok(h->dtype) || !block_ok(h->block) || h->n == 0 || h->n > kMaxValues) return SZX_ERR_INVALID;
    if (h->tile_blocks != tile_blocks(h->block, width(h->dtype))) return SZX_ERR_INVALID;
    const Geometry g = make_geometry(h->n, h->block, width(h->dtype));
    if (h->total_bytes > in_bytes || h->total_bytes < g.off_rec) return SZX_ERR_CORRUPT;
    if (out_capacity < h->n * width(h->dtype)) return SZX_ERR_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    return from_cuda(launch_decompress(d_in, in_bytes, h->total_bytes, h->n, (int)h->dtype, h->block, d_out,
                                       d_status, true, s, 0, ~0ull, clear));
}

}  // namespace szx

extern "C" {

size_t szx_stream_max_bytes(size_t n, szx_dtype dtype, uint32_t block) {
    if (!dtype_ok(dtype) || !block_ok(block) || n == 0 || n > kMaxValues) return 0;
    return (size_t)stream_max(n, block, width(dtype));
}

size_t szx_compress_bound(size_t n, szx_dtype dtype, uint32_t block) {
    const size_t smax = szx_stream_max_bytes(n, dtype, block);
    if (!smax) return 0;
    const Geometry g = make_geometry(n, block, width(dtype));
    return (size_t)(align256(smax) + workspace_bytes(g.ntiles));
}

szx_status szx_compress_async(const void *d_in, size_t n, szx_dtype dtype, double eb, uint32_t block,
                              void *d_out, size_t out_capacity, uint64_t *d_result, szx_stream_t stream) {
    return compress_async_with(d_in, n, dtype, eb, block, d_out, out_capacity, d_result, stream, Clear::automatic);
}

szx_status szx_compress(const void *d_in, size_t n, szx_dtype dtype, double eb, uint32_t block, void *d_out,
                        size_t out_capacity, size_t *out_bytes, szx_stream_t stream) {
    if (!out_bytes) return SZX_ERR_INVALID;
    szx_status st = szx_compress_async(d_in, n, dtype, eb, block, d_out, out_capacity, nullptr, stream);
    if (st != SZX_OK) return st;
    const uint64_t ws = align256(stream_max(n, block, width(dtype)));
    const Workspace *w = reinterpret_cast<const Workspace *>(static_cast<const uint8_t *>(d_out) + ws);
    unsigned long long result[2] = {0, 0};
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(result, &w->result, sizeof(result), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SZX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZX_ERR_CUDA;
    if (result[1] != 0) return (szx_status)result[1];
    *out_bytes = (size_t)result[0];
    return SZX_OK;
}

szx_status szx_header_read(const void *d_in, size_t in_bytes, szx_header *h, szx_stream_t stream) {
    if (!d_in || !h) return SZX_ERR_INVALID;
    if (in_bytes < (size_t)kHeaderBytes) return SZX_ERR_CORRUPT;
    uint8_t buf[kHeaderBytes];
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(buf, d_in, kHeaderBytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SZX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZX_ERR_CUDA;
    return parse_header(buf, in_bytes, h);
}

szx_status szx_decompress_async(const void *d_in, size_t in_bytes, const szx_header *h, void *d_out,
                                size_t out_capacity, uint32_t *d_status, szx_stream_t stream) {
    return decompress_async_with(d_in, in_bytes, h, d_out, out_capacity, d_status, stream, Clear::automatic);
}

szx_status szx_decompress_range_async(const void *d_in, size_t in_bytes, const szx_header *h, size_t first_block,
                                      size_t nblocks, void *d_out, size_t out_capacity, uint32_t *d_status,
                                      szx_stream_t stream) {
    if (!d_in || !h || !d_out) return SZX_ERR_INVALID;
    if (!aligned16(d_in) || !aligned16(d_out)) return SZX_ERR_INVALID;
    if (!dtype_ok(h->dtype) || !block_ok(h->block) || h->n == 0 || h->n > kMaxValues) return SZX_ERR_INVALID;
    if (h->tile_blocks != tile_blocks(h->block, width(h->dtype))) return SZX_ERR_INVALID;
    const Geometry g = make_geometry(h->n, h->block, width(h->dtype));
    if (h->total_bytes > in_bytes || h->total_bytes < g.off_rec) return SZX_ERR_CORRUPT;
    if (nblocks == 0 || first_block >= g.nb || nblocks > g.nb - first_block) return SZX_ERR_INVALID;
    const uint64_t last = first_block + nblocks;
    const uint64_t vals = min_u64(h->n, last * h->block) - (uint64_t)first_block * h->block;
    if (out_capacity < vals * width(h->dtype)) return SZX_ERR_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    return from_cuda(launch_decompress(d_in, in_bytes, h->total_bytes, h->n, (int)h->dtype, h->block, d_out,
                                       d_status, true, s, first_block, last));
}

szx_status szx_decompress(const void *d_in, size_t in_bytes, void *d_out, size_t out_capacity, size_t *n_out,
                          szx_dtype *dtype_out, szx_stream_t stream) {
    szx_header h;
    szx_status st = szx_header_read(d_in, in_bytes, &h, stream);
    if (st != SZX_OK) return st;
    if (n_out) *n_out = (size_t)h.n;
    if (dtype_out) *dtype_out = h.dtype;
    if (!d_out) return SZX_ERR_INVALID;
    uint32_t *slot = status_slot(&st);
    if (!slot) return st;
    st = szx_decompress_async(d_in, in_bytes, &h, d_out, out_capacity, slot, stream);
    if (st != SZX_OK) return st;
    uint32_t code = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&code, slot, sizeof(code), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SZX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZX_ERR_CUDA;
    return (szx_status)code;
}

const char *szx_status_string(szx_status s) {
    switch (s) {
        case SZX_OK: return "ok";
        case SZX_ERR_INVALID: return "invalid argument";
        case SZX_ERR_TOO_SMALL: return "output buffer too small";
        case SZX_ERR_CORRUPT: return "corrupt or truncated stream";
        case SZX_ERR_NOMEM: return "out of host memory";
        case SZX_ERR_CUDA: return "CUDA runtime error";
        case SZX_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *szx_version(void) { return "szx-b300 1.0 (sm_103a)"; }

}  // extern "C"
