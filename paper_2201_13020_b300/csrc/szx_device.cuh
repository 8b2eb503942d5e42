// szx_device.cuh -- device-side building blocks of the sm_103a SZx codec.
//
// Formats, the exact |a - b| <= e test, warp reductions/scans, inline PTX for
// the Blackwell bulk-copy engine (cp.async.bulk + mbarrier), and the stream
// geometry shared by the compress and decompress kernels.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace szx {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kMagic = 0x42585A53u;  // "SZXB"
constexpr uint32_t kVersion = 1;
constexpr int kHeaderBytes = 64;
constexpr int kWarps = 8;  // warps per CTA in both kernels
constexpr int kThreads = kWarps * 32;

// Block kinds (Algorithm 1: constant / non-constant; plus verbatim "raw").
enum : uint8_t { kConst = 0, kNonConst = 1, kRaw = 2 };

// Device error bits (compress workspace and decompress status word).
// kErrTimeout: the offset look-back gave up; kErrTmaTimeout: a bulk or
// tensor copy did not complete within its wait limit.
enum : uint32_t { kErrTimeout = 1u, kErrCorrupt = 2u, kErrTmaTimeout = 4u, kErrInternal = 8u };

// ---------------------------------------------------------------------------
// IEEE formats

template <typename T>
struct Fmt;

template <>
struct Fmt<float> {
    using U = uint32_t;
    using S = int32_t;
    static constexpr int w = 4, W = 32, E = 8, M = 23, bias = 127;
    __device__ __forceinline__ static float from(U u) { return __uint_as_float(u); }
    __device__ __forceinline__ static U bits(float f) { return __float_as_uint(f); }
    __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ __forceinline__ static float half(float a) { return __fmul_rn(a, 0.5f); }
    __device__ __forceinline__ static int clz(U x) { return __clz(x); }
    __device__ __forceinline__ static bool finite(U u) { return ((u >> 23) & 0xFFu) != 0xFFu; }
    __device__ __forceinline__ static int expo(U u) { return (int)((u >> 23) & 0xFFu) - 127; }
    // order-preserving signed key: totalOrder on finite values (-0 < +0)
    __device__ __forceinline__ static S key(U u) { return (S)(u ^ ((U)((S)u >> 31) & 0x7FFFFFFFu)); }
    __device__ __forceinline__ static U unkey(S k) { return (U)k ^ ((U)(k >> 31) & 0x7FFFFFFFu); }
    static constexpr S kKeyPosInf = 0x7F800000;
    static constexpr S kKeyNegInf = (S)0x807FFFFF;
};

template <>
struct Fmt<double> {
    using U = uint64_t;
    using S = int64_t;
    static constexpr int w = 8, W = 64, E = 11, M = 52, bias = 1023;
    __device__ __forceinline__ static double from(U u) { return __longlong_as_double((long long)u); }
    __device__ __forceinline__ static U bits(double f) { return (U)__double_as_longlong(f); }
    __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ __forceinline__ static double half(double a) { return __dmul_rn(a, 0.5); }
    __device__ __forceinline__ static int clz(U x) { return __clzll((long long)x); }
    __device__ __forceinline__ static bool finite(U u) { return ((u >> 52) & 0x7FFull) != 0x7FFull; }
    __device__ __forceinline__ static int expo(U u) { return (int)((u >> 52) & 0x7FFull) - 1023; }
    __device__ __forceinline__ static S key(U u) {
        return (S)(u ^ ((U)((S)u >> 63) & 0x7FFFFFFFFFFFFFFFull));
    }
    __device__ __forceinline__ static U unkey(S k) {
        return (U)k ^ ((U)(k >> 63) & 0x7FFFFFFFFFFFFFFFull);
    }
    static constexpr S kKeyPosInf = 0x7FF0000000000000ll;
    static constexpr S kKeyNegInf = (S)0x800FFFFFFFFFFFFFull;
};

// Mask of the top 8q bits of a W-bit word (q in [1, W/8]).
template <typename U>
__device__ __forceinline__ U top_bytes_mask(int q) {
    constexpr int W = 8 * sizeof(U);
    return q * 8 >= W ? ~(U)0 : ~(U)0 << (W - 8 * q);
}

// Exact |a - b| <= e for finite a, b and finite e >= 0 (Eq. 1 as an exact
// predicate).  RN(a - b) decides every case except |RN(a - b)| == e, where the
// sign of the rounding error, recovered exactly by Knuth's TwoSum, decides.
template <typename T>
__device__ __forceinline__ bool within(T a, T b, T e) {
    using F = Fmt<T>;
    using U = typename F::U;
    T s = F::sub(a, b);
    // |s| against e on the IEEE bit patterns, which order the non-negative
    // values (and place NaNs above infinity); integer compares, not
    // floating-point ones, which are slow for f64
    const U as = F::bits(s) & ~(U(1) << (F::W - 1));
    const U eb = F::bits(e);
    if (as < eb) return true;
    if (as != eb) return false;  // > e, NaN, or an overflow to infinity
    T y = -b;
    T bv = F::sub(s, a);
    T av = F::sub(s, bv);
    T t = F::add(F::sub(a, av), F::sub(y, bv));
    if (s > T(0)) return t <= T(0);
    if (s < T(0)) return t >= T(0);
    return t == T(0);
}

// ---------------------------------------------------------------------------
// warp helpers

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__host__ __device__ __forceinline__ uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// Exclusive prefix sum over the warp; *total receives the warp's sum.
template <typename V>
__device__ __forceinline__ V warp_exclusive_scan(V v, V *total) {
    const int lane = lane_id();
    V x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        V y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    *total = __shfl_sync(kFull, x, 31);
    return x - v;
}

// ---------------------------------------------------------------------------
// Blackwell bulk-copy engine (TMA, non-tensor form) and mbarriers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

// A kernel launched as the programmatic dependent of the one before it on the
// stream may start while that one still runs: every thread calls this before
// its first global-memory access, and it returns once the earlier kernels have
// finished and their writes are visible (at once for a plain launch).
__device__ __forceinline__ void wait_prior_grids() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One probe of an mbarrier phase; the thread may be suspended for up to about
// 1 us (suspend-time hint) while the phase is pending.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}

// Wait on an mbarrier phase for at most limit_ns of wall time; returns false
// if the deadline passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait_hint(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// global -> shared bulk copy, completion counted on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// shared -> global bulk copy (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_addr(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Make generic-proxy shared-memory writes visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Look-back words carry their whole payload (flag and count in one 64-bit
// word), so relaxed (single-copy atomic) accesses suffice: no other data is
// published through them.
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------------------
// stream geometry (host and device)

__host__ __device__ __forceinline__ uint64_t pad16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

__host__ __device__ constexpr uint32_t tile_blocks(uint32_t b, uint32_t w) {
    uint32_t g = 32768u / (b * w);
    return g < 8 ? 8 : g;
}

struct Geometry {
    uint64_t n, nb, ntiles;
    uint32_t b, G, w;
    uint64_t off_state, off_mu, off_index, off_rec;
};

__host__ __device__ inline Geometry make_geometry(uint64_t n, uint32_t b, uint32_t w) {
    Geometry g;
    g.n = n;
    g.b = b;
    g.w = w;
    g.G = tile_blocks(b, w);
    g.nb = (n + b - 1) / b;
    g.ntiles = (g.nb + g.G - 1) / g.G;
    g.off_state = kHeaderBytes;
    g.off_mu = g.off_state + pad16((g.nb + 7) / 8);
    g.off_index = g.off_mu + pad16(g.nb * w);
    g.off_rec = g.off_index + pad16((g.ntiles + 1) * 8);
    return g;
}

// Largest record of one tile: every block raw.
__host__ __device__ __forceinline__ uint32_t record_max_bytes(uint32_t G, uint32_t b, uint32_t w) {
    return (uint32_t)pad16((uint64_t)G * (b / 4 + 1) + (uint64_t)G * b * w);
}

// Compress workspace, at the 256-byte-aligned end of the largest stream.
struct Workspace {
    uint32_t ticket;  // next tile ticket (tiles are processed in ticket order)
    uint32_t done;    // tiles finished
    uint32_t err;     // kErr* bits
    uint32_t reserved0;     // zero (a copy that does not complete sets kErrTmaTimeout in err)
    unsigned long long nn, nraw, nesc;
    unsigned long long result[2];  // stream bytes, status (written by the last tile)
    unsigned long long lookback_timeouts;  // tiles whose look-back gave up
    uint32_t reserved1;       // zero
    uint32_t first_lb_tile;   // 1 + the first tile whose look-back timed out
    uint32_t first_bad_tile;  // 1 + the first tile that failed a self-check
    uint32_t bad_code;        // which self-check failed
    uint32_t diag[12];
    // followed by ntiles look-back words
};
constexpr uint64_t kWsHeader = 128;
static_assert(sizeof(Workspace) == kWsHeader, "workspace header layout");

// look-back word: 2-bit flag | 62-bit record byte count
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

__host__ __device__ __forceinline__ uint64_t workspace_bytes(uint64_t ntiles) {
    return kWsHeader + 8 * ntiles;
}

// One field of a compression launch.  A launch covers one field (passed by
// value) or a table of fields of the same dtype and block length in device
// memory; its tiles form one global list, field after field.
struct alignas(64) CField {
    CUtensorMap tmap;  // the field's input rows (TMA), valid if use_tma
    const uint8_t *in;
    uint8_t *out;
    Workspace *ws;  // the field's counters and result
    uint64_t *lookback;  // the field's look-back words (one per tile, zeroed)
    uint64_t *d_result;  // {stream bytes, status} on completion, or null
    Geometry g;
    uint64_t e_bits;
    uint64_t rows_full;  // 128-byte input rows fully inside the input
    uint64_t tile0;      // the field's first tile in the launch's global list
    uint32_t dtype;
    uint32_t use_tma;
};


// One field of a decompression launch (same arrangement as CField).
struct alignas(64) DField {
    CUtensorMap tmap;  // the field's output rows (one box per decoding warp), valid if use_tma
    const uint8_t *in;  // the stream
    uint8_t *out;       // n values
    uint32_t *status;   // szx_status, folded in with atomicMax, or null
    Geometry g;
    uint64_t rec_total;    // bytes of the tile records
    uint64_t total_bytes;  // stream size (the header's)
    uint64_t rows_full;    // 128-byte output rows fully inside the output
    uint64_t tile0;        // the field's first tile in the launch's global list
    uint64_t tile_lo;      // the first tile decoded (a block range starts there)
    uint64_t blk_lo, blk_hi;  // blocks written: out holds values from block blk_lo on
    uint64_t row_lo;       // blk_lo's first 128-byte row (rows of out count from it)
    uint32_t dtype;
    uint32_t check_header;  // re-check the stream header on the device
    uint32_t use_tma;
};

}  // namespace szx
