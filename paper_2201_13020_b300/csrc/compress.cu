// compress.cu -- single-pass SZx compression kernel for sm_103a.
//
// Persistent, warp-specialised CTAs take tiles of G consecutive blocks (32
// KiB of input) by ticket and turn each into the tile's record.  Tickets are
// processed in the order they were taken, so the decoupled look-back over
// tile record sizes -- the device-wide exclusive scan that places each record
// (the prefix scan of Sec. V-B) -- only ever waits on tiles that are running
// or done.
//
// Work layout: every lane owns 128 contiguous input bytes (32 f32 or 16 f64
// values); a block of b values is handled by LPB = b / VPL adjacent lanes (4
// lanes for f32, b = 128).  The serial previous-value dependency stays inside
// a lane except at lane boundaries.
//
// Per CTA: a ring of three tile buffers and three roles.  A producer thread
// takes tickets and copies tiles in with the TMA unit (2-D tensor copy, rows
// of 128 B, 128-byte swizzle, so that each lane reads its row without bank
// conflicts); it takes a tile's ticket only once the consumers are on the tile
// before it, which keeps the look-back waits short.  Eight consumer warps
// encode a tile and build its record in place; a storer warp places and
// stores records.  The roles hand stages to
// each other through mbarriers (full / encoded / ready / empty), so encoding
// never waits for a look-back or a store, and every wait is bounded.  The
// same kernel serves one field (its descriptor is a kernel parameter) and
// batches (a table of descriptors in device memory, BATCH).  Tiles wholly
// inside the input run a copy of the per-tile work compiled for full blocks.
// Per tile:
//   1. each consumer warp loads its rows and clears them (the buffer becomes
//      the record), then encodes in registers -- block statistics
//      (Algorithm 1): NaN-propagating min/max per lane, reduced over the
//      block's lanes with shuffles; mu, r, the exact constant test, reqBits
//      (Eq. 4) -- for one f64 field with 128 <= b <= 512 computed by warp 0 for every
//      block of the tile from the keys the warps hand in through shared
//      memory -- then the Eq. 5 shift and truncation.  The per-value bound check is
//      skipped when a block-level bound proves it passes (see
//      bound_check_needed); otherwise a fast test runs and an exact slow path
//      re-checks a block that fails it, raising reqBits while a value exceeds
//      e.  Then the identical-leading-byte codes against the previous value
//      (from each word's top 32 bits: the position of the top set bit of the
//      xor gives the code) and the lanes' mid-byte counts.  The
//      warp writes its blocks' mu values, publishes its totals and forms its
//      lanes' plane counts;
//   2. the warps meet once (an mbarrier); warp reductions of the warps'
//      totals give every block its rank and mid-byte offset; warp 0 publishes
//      the tile's record size for the look-back;
//   3. lanes write lead codes, reqBits bytes and the mid-byte planes (plane j
//      = byte j of every value whose code is <= j, ascending index): a 4x4
//      byte transpose of four values gives their byte-j word, a 256-entry
//      table compacts the selected bytes, and shared-memory OR writes place the
//      run at its bit offset (two funnel shifts).  When every lane of a warp
//      keeps byte 2 of all its values (no code 3), plane 2 goes out as whole
//      words, each one funnel shift of two consecutive groups, with plain
//      stores and an OR for the two edge words only;
//   4. the storer finishes the look-back, writes the tile index entry and
//      bulk-stores the record (cp.async.bulk) to its offset, writing the
//      tile's state bits and counts while the store reads; once it has read
//      the buffer, the producer refills it.  The last CTA to finish writes
//      each field's header.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <limits>
#include <mutex>
#include <type_traits>

#include "szx_device.cuh"
#include "szx_launch.h"

#ifndef SZX_CHECKS
#define SZX_CHECKS 0  // 1: self-checks of every record write (diagnostic builds)
#endif

namespace szx {

struct CompressLaunch {
    const CField *fields;  // device table of nfields fields, or null: the single field
    uint32_t nfields;
    uint64_t total_tiles;
    uint32_t *ticket;  // launch counters, zeroed before the launch
    uint32_t *done;
    uint32_t *err;     // launch-wide kErr* bits (folded into every field's status)
    uint64_t lookback_ns;  // wall-time limit of the look-back wait
    uint64_t copy_ns;      // wall-time limit of a tile copy wait
};

template <bool BATCH>
__device__ __forceinline__ const CField *field_ptr(const CField &one, const CompressLaunch &lc, uint32_t f) {
    if constexpr (BATCH) return lc.fields + f;
    else return &one;  // the kernel parameter itself (param space)
}

// The field holding global tile t: the last one whose first tile is <= t.
template <bool BATCH>
__device__ __forceinline__ uint32_t field_of(const CompressLaunch &lc, uint64_t t) {
    if constexpr (!BATCH) return 0;
    uint32_t lo = 0, hi = lc.nfields - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (lc.fields[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// compaction table: for the 2-bit codes of four values (value k at bits 2k),
// one 16-byte entry whose word j (j = 0..2; word 3 repeats word 2) is the
// byte-permute selector taking, in order, the bytes of the values whose code
// is <= j (unused nibbles select zero), plus the number of such values << 16.
// Built at compile time.

struct PlaneLut {
    uint32_t v[1024];
};
constexpr PlaneLut make_plane_lut() {
    PlaneLut t{};
    for (uint32_t i = 0; i < 1024; ++i) {
        const uint32_t j = (i & 3u) < 2u ? (i & 3u) : 2u, code = i >> 2;
        uint32_t sel = 0x4444u, cnt = 0;
        for (uint32_t k = 0; k < 4; ++k) {
            if (((code >> (2 * k)) & 3u) <= j) {
                sel = (sel & ~(0xFu << (4 * cnt))) | (k << (4 * cnt));
                ++cnt;
            }
        }
        t.v[i] = sel | ((cnt * 8) << 16);
    }
    return t;
}
__device__ const PlaneLut kPlaneLut = make_plane_lut();

// ---------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ float min_nan(float a, float b) {
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float max_nan(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// three-input forms (one instruction for two values)
__device__ __forceinline__ float min3_nan(float a, float b, float c) {
    float r;
    asm("min.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max3_nan(float a, float b, float c) {
    float r;
    asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) { return __byte_perm(a, b, s); }

// Position (0..31) of the most significant set bit of a nonzero word.
__device__ __forceinline__ uint32_t top_bit(uint32_t x) {
    uint32_t f;
    asm("bfind.u32 %0, %1;" : "=r"(f) : "r"(x));
    return f;
}

// OR a run of up to 4 bytes (little-endian in `run`, zero above its length)
// into the zero-initialised byte buffer at bit offset pb (a multiple of 8).
__device__ __forceinline__ void or_bytes(uint32_t *words, uint32_t pb, uint32_t run) {
    // the two words of (uint64_t)run << (pb mod 32), by funnel shifts (which
    // take the shift modulo 32 themselves)
    uint32_t *wp = words + (pb >> 5);
    atomicOr(wp, __funnelshift_l(0u, run, pb));
    const uint32_t hi = __funnelshift_l(run, 0u, pb);
    if (hi) atomicOr(wp + 1, hi);  // OR-ing zeros would change nothing
}

// Record a failed self-check (first tile and check id).
__device__ __forceinline__ void report_bad(Workspace *ws, uint32_t tile, uint32_t code) {
    atomicOr(&ws->err, kErrInternal);
    if (atomicCAS(&ws->first_bad_tile, 0u, tile + 1) == 0u) ws->bad_code = code;
}

// 4x4 byte transpose: W[j] holds byte j (most significant first) of the four
// 32-bit words t0..t3, value k in byte k.
__device__ __forceinline__ void transpose4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, uint32_t (&W)[4]) {
    const uint32_t a = prmt(t0, t1, 0x5140), b = prmt(t0, t1, 0x7362);
    const uint32_t c = prmt(t2, t3, 0x5140), d = prmt(t2, t3, 0x7362);
    W[3] = prmt(a, c, 0x5410);
    W[2] = prmt(a, c, 0x7632);
    W[1] = prmt(b, d, 0x5410);
    W[0] = prmt(b, d, 0x7632);
}

// Effective exponent: the unbiased exponent, with subnormals and zero at the
// minimum normal exponent (their spacing is 2^(emin - M)).
template <typename T>
__device__ __forceinline__ int eff_expo(typename Fmt<T>::U u) {
    using F = Fmt<T>;
    const int f = (int)((u >> F::M) & ((1u << F::E) - 1));
    return (f ? f : 1) - F::bias;
}

// Does the per-value check |d - RN(v' + mu)| <= e need to run at reqBits =
// 1 + E + R?  It can be skipped when a block-level bound proves every value
// passes (the result is then the same as running it):
//   For d in [mn, mx], v = RN(d - mu) has |v| <= max(|RN(mn - mu)|,
//   |RN(mx - mu)|), so its effective exponent is at most P.  Truncating v to R
//   mantissa bits drops less than 2^(p(v) - R) minus one unit of v, and the
//   rounding of v adds at most half a unit, so |v' + mu - d| < 2^(P - R) = C.
//   Then |v' + mu| < B + C with B = max(|mn|, |mx|), so both lie below
//   2^(K + 2), K = max(p(B), P - R), where half a spacing is at most
//   2^(K - M) = U; hence |d - d'| < C + U.  If C + U <= e, every value passes.
// The comparison is done exactly in integers on e's significand.  K is kept
// three binades below the largest exponent so that nothing overflows.
template <typename T>
__device__ __forceinline__ bool bound_check_needed(T mn, T mx, T mu, int R, typename Fmt<T>::U e_bits) {
    using F = Fmt<T>;
    using U = typename F::U;
    const int P = max(eff_expo<T>(F::bits(F::sub(mx, mu))), eff_expo<T>(F::bits(F::sub(mn, mu))));
    const U babs = max(F::bits(mn) & ~(U(1) << (F::W - 1)), F::bits(mx) & ~(U(1) << (F::W - 1)));
    const int a = P - R;
    const int K = max(eff_expo<T>(babs), a);
    if (K > (1 << (F::E - 1)) - 1 - 3) return true;  // near overflow: check
    const int ee = eff_expo<T>(e_bits);
    const U efield = (e_bits >> F::M) & ((U(1) << F::E) - 1);
    const U me = (e_bits & ((U(1) << F::M) - 1)) | (efield ? (U(1) << F::M) : U(0));  // e = me * 2^(ee - M)
    if (me == 0) return true;
    const int A = a - ee + F::M, V = K - F::M - ee + F::M;  // C = 2^A, U = 2^V in units of 2^(ee - M)
    if (A > F::M + 1 || V > F::M + 1) return true;
    const unsigned long long m = (unsigned long long)me;
    bool fits;
    if (A >= 0 && V >= 0) fits = (1ull << A) + (1ull << V) <= m;
    else if (A >= 0) fits = (1ull << A) < m;
    else if (V >= 0) fits = (1ull << V) < m;
    else fits = true;  // both below one unit of e's significand, and me >= 1
    return !fits;
}

// ---------------------------------------------------------------------------
// per-lane encoding (step 1); FULL: every value of the lane is valid

// One block's statistics from its min / max keys (Algorithm 1): r =
// RN(RN(mx - mn) / 2), mu = RN(mn + r), the class (raw when a value or r or mu
// is not finite; constant by the exact test |d - mu| <= e at both extremes),
// R of Eq. 4 and reqBits = 1 + E + R before any escalation.
template <typename T>
struct BlockStats {
    T mn, mx, mu;
    int kind, R, req0;
};
template <typename T>
__device__ __forceinline__ BlockStats<T> block_stats(typename Fmt<T>::S kmn, typename Fmt<T>::S kmx, bool exists,
                                                     T e) {
    using F = Fmt<T>;
    BlockStats<T> o;
    // a NaN's key lies above +inf (or, for f64 negative NaNs, below -inf)
    const bool all_finite = kmn > F::kKeyNegInf && kmn < F::kKeyPosInf && kmx > F::kKeyNegInf &&
                            kmx < F::kKeyPosInf;
    o.mn = F::from(F::unkey(kmn));
    o.mx = F::from(F::unkey(kmx));
    const T r = F::half(F::sub(o.mx, o.mn));
    o.mu = F::add(o.mn, r);
    o.kind = kConst;
    if (!exists) o.kind = 0xFF;
    else if (!all_finite || !F::finite(F::bits(r)) || !F::finite(F::bits(o.mu))) o.kind = kRaw;
    else if (!(within(o.mx, o.mu, e) && within(o.mn, o.mu, e))) o.kind = kNonConst;
    int R = F::expo(F::bits(r)) - F::expo(F::bits(e));
    o.R = R < 0 ? 0 : (R > F::M ? F::M : R);
    o.req0 = 1 + F::E + o.R;
    return o;
}

// A block's statistics as the tile's statistics warp hands them out (XS).
template <typename T>
struct XOut {
    T mu;
    int kind, req0;
    bool check;
};

// XS: the block statistics come from xchg(kmn, kmx, XOut&) -- one warp
// computes them for every block of the tile -- instead of from this lane;
// false when that exchange ran out of time.
template <typename T, int LPB, int VPL, bool FULL, bool XS, typename Xchg>
__device__ __forceinline__ bool encode_lane(typename Fmt<T>::U (&x)[VPL], uint32_t (&codes)[(2 * VPL + 31) / 32],
                                            int &kind, int &req, int &req0, T &mu_out, uint32_t &mk_out,
                                            const typename Fmt<T>::U *src, int nvalid, bool exists, T e,
                                            uint64_t e_bits, Workspace *ws, uint32_t tile, Xchg &&xchg) {
    using F = Fmt<T>;
    using U = typename F::U;
    using S = typename F::S;
    constexpr int w = F::w;
    constexpr int W = F::W;
    constexpr int NCODE = (2 * VPL + 31) / 32;
    const int lane = lane_id();
    const int sub = lane % LPB;

    // min / max (NaN and infinities propagate, so one test finds them)
    S kmn = std::numeric_limits<S>::max(), kmx = std::numeric_limits<S>::min();
    if constexpr (sizeof(T) == 4) {
        float lmn = F::from(x[0]), lmx = F::from(x[0]);
        if constexpr (FULL && VPL % 2 == 0) {
#pragma unroll
            for (int m = 1; m + 1 < VPL; m += 2) {
                lmn = min3_nan(lmn, F::from(x[m]), F::from(x[m + 1]));
                lmx = max3_nan(lmx, F::from(x[m]), F::from(x[m + 1]));
            }
            lmn = min_nan(lmn, F::from(x[VPL - 1]));
            lmx = max_nan(lmx, F::from(x[VPL - 1]));
        } else {
#pragma unroll
            for (int m = 1; m < VPL; ++m) {
                if (FULL || m < nvalid) {
                    lmn = min_nan(lmn, F::from(x[m]));
                    lmx = max_nan(lmx, F::from(x[m]));
                }
            }
        }
        if (FULL || nvalid > 0) {
            kmn = F::key(F::bits(lmn));
            kmx = F::key(F::bits(lmx));
        }
    } else {
#pragma unroll
        for (int m = 0; m < VPL; ++m) {
            if (FULL || m < nvalid) {
                const S kx = F::key(x[m]);
                kmn = kx < kmn ? kx : kmn;
                kmx = kx > kmx ? kx : kmx;
            }
        }
    }
#pragma unroll
    for (int d = 1; d < LPB; d <<= 1) {
        const S omn = __shfl_xor_sync(kFull, kmn, d), omx = __shfl_xor_sync(kFull, kmx, d);
        kmn = omn < kmn ? omn : kmn;
        kmx = omx > kmx ? omx : kmx;
    }
    T mn, mx, mu;
    int R = 0;
    bool check_x = false;
    if constexpr (XS) {
        XOut<T> o;
        if (!xchg(kmn, kmx, o)) return false;
        mu = o.mu;
        mn = mx = mu;  // used only by the block-level bound, already decided
        kind = o.kind;
        req0 = o.req0;
        check_x = o.check;
    } else {
        const BlockStats<T> bs = block_stats<T>(kmn, kmx, exists, e);
        mn = bs.mn;
        mx = bs.mx;
        mu = bs.mu;
        kind = bs.kind;
        R = bs.R;
        req0 = bs.req0;
    }
    mu_out = mu;
    req = req0;
    if (__all_sync(kFull, kind != kNonConst)) {
        // no block of the warp keeps truncated values (all constant, raw or
        // absent): truncation, bound checks and lead codes would go unused
#pragma unroll
        for (int i = 0; i < NCODE; ++i) codes[i] = 0;
        mk_out = kind == kRaw ? (uint32_t)nvalid * w : 0u;
        return true;
    }
    const bool check = XS ? check_x : kind == kNonConst && bound_check_needed<T>(mn, mx, mu, R, (U)e_bits);

    // truncation; with `check`, a fast test of every value (one rounding)
    bool ok = true;
    {
        const int s = (8 - (req & 7)) & 7;
        const U mask = top_bytes_mask<U>((req + s) >> 3);
        if (check) {
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                if (FULL || m < nvalid) {
                    const T xv = F::from(x[m]);
                    const U t = (F::bits(F::sub(xv, mu)) >> s) & mask;
                    const T dp = F::add(F::from((U)(t << s)), mu);
                    ok = ok && fabs(F::sub(xv, dp)) < e;
                    x[m] = t;
                }
            }
        } else {
            // the bytes below the top q are left in place: lead codes stop at
            // min(q, 3) bytes and the packing takes bytes 0..q-1 only, so they
            // never matter (only a decoded value, as in the check above, needs
            // the masked word)
#pragma unroll
            for (int m = 0; m < VPL; ++m)
                if (FULL || m < nvalid) x[m] = F::bits(F::sub(F::from(x[m]), mu)) >> s;
        }
    }
    const uint32_t segmask = (LPB == 32 ? kFull : ((1u << LPB) - 1u)) << (lane & ~(LPB - 1));
    {
        const uint32_t bal = __ballot_sync(kFull, ok || kind != kNonConst);
        ok = (bal & segmask) == segmask;
    }
    // exact slow path: ties with e and real failures (reqBits grows, or the
    // block is stored raw at full width)
    bool pending = kind == kNonConst && !ok;
    if (pending && sub == 0) atomicAdd(&ws->diag[0], 1u);
    int rounds = 0;
    while (__any_sync(kFull, pending)) {
        if (SZX_CHECKS && ++rounds > W) {  // reqBits rises one bit a round, at most to W
            if (lane == 0) report_bad(ws, tile, 3);
            if (pending) kind = kRaw;
            break;
        }
        bool ok2 = true;
        if (pending) {
            const int s = (8 - (req & 7)) & 7;
            const U mask = top_bytes_mask<U>((req + s) >> 3);
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                if (m < nvalid) {
                    // the lane's input values (its shared-memory rows are
                    // already cleared for the record): re-read from global
                    const T xv = F::from(src[m]);
                    const U t = (F::bits(F::sub(xv, mu)) >> s) & mask;
                    ok2 = ok2 && within(xv, F::add(F::from((U)(t << s)), mu), e);
                    x[m] = t;
                }
            }
        }
        const uint32_t bal = __ballot_sync(kFull, ok2);
        if (pending) {
            if ((bal & segmask) == segmask) {
                pending = false;
            } else if (++req > W) {
                kind = kRaw;
                pending = false;
            }
        }
    }

    // identical-leading-byte codes against the previous truncated word
    const int s = (8 - (req & 7)) & 7;
    const int q = (req + s) >> 3;
    const int lmax = q < 3 ? q : 3;
#pragma unroll
    for (int i = 0; i < NCODE; ++i) codes[i] = 0;
    {
        // Only the top lmax <= 3 bytes decide a code, and they lie in the
        // word's top 32 bits: the count runs on those (one 32-bit xor and
        // clz per value, also for f64)
        uint32_t prev = (uint32_t)(__shfl_up_sync(kFull, x[VPL - 1], 1) >> (W - 32));
        if (sub == 0) prev = 0;
        // a set bit in byte lmax (counted from the top) caps the count at lmax
        const uint32_t cap = 1u << (31 - 8 * lmax);
        if constexpr (FULL) {
            // f = the position of the top set bit of (xor | cap); the code is
            // 3 - (f >> 3), the complement of f's bits 3-4.  Shifting f so
            // that those bits land on the code's place 2k (k = m mod 16)
            // leaves f's bits 0-2 just below it; values with the same k mod 4
            // go to one word, 8 bits apart, where those bits never reach
            // another code (so adding is OR-ing: one shift-add per value), and
            // one mask per word keeps the codes alone
            uint32_t acc[NCODE][4];
#pragma unroll
            for (int i = 0; i < NCODE; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0;
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                const uint32_t top = (uint32_t)(x[m] >> (W - 32));
                const uint32_t f = top_bit((top ^ prev) | cap);
                const int p = 2 * (m & 15) - 3;
                acc[m >> 4][m & 3] += p >= 0 ? (f << p) : (f >> -p);
                prev = top;
            }
#pragma unroll
            for (int i = 0; i < NCODE; ++i)
                codes[i] = ~((acc[i][0] & 0x03030303u) | (acc[i][1] & 0x0C0C0C0Cu) | (acc[i][2] & 0x30303030u) |
                             (acc[i][3] & 0xC0C0C0C0u));
        } else {
            // each value's code in its own word first, then an OR tree (no
            // serial chain through the code words)
            uint32_t part[VPL];
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                const uint32_t top = (uint32_t)(x[m] >> (W - 32));
                int l = __clz((top ^ prev) | cap) >> 3;
                if (m >= nvalid) l = 0;
                part[m] = (uint32_t)l << (2 * (m & 15));
                prev = top;
            }
#pragma unroll
            for (int d = 1; d < 16; d <<= 1) {
#pragma unroll
                for (int m = 0; m + d < VPL; m += 2 * d) part[m] |= part[m + d];
            }
#pragma unroll
            for (int i = 0; i < NCODE; ++i) codes[i] = part[16 * i];
        }
    }
    uint32_t suml = 0;
#pragma unroll
    for (int i = 0; i < NCODE; ++i) suml += __popc(codes[i] & 0x55555555u) + 2 * __popc(codes[i] & 0xAAAAAAAAu);
    // this lane's mid bytes (raw: its verbatim bytes)
    mk_out = kind == kNonConst ? (uint32_t)(nvalid * q) - suml : (kind == kRaw ? (uint32_t)nvalid * w : 0u);
    return true;
}

// Shared-memory layout of the compress kernel: kStages tile buffers (each
// later reused for its tile's record), per-stage block metadata, the table.
constexpr int kStages = 3;
// A CTA has NW consumer warps (8 or 4), then the producer and the storer
// warp.  The tile (G blocks, a fixed number of 128-byte rows) is laid out over
// the consumers' lanes, each lane taking RPL = rows / (32 NW) consecutive rows:
// with fewer warps a lane holds more values and a warp more blocks.
__host__ __device__ constexpr int compress_threads(int nw) { return nw * 32 + 64; }

struct CSmem {
    uint32_t buf_stride, buf_bytes;  // tile buffer st at st * buf_stride (1024-aligned)
    uint32_t meta0, meta_stride;     // metadata block st at meta0 + st * meta_stride
    uint32_t m_kind, m_w;  // offsets inside a metadata block: block kinds, per-warp totals
    uint32_t lut, xs, total;
};
__host__ __device__ inline CSmem compress_smem(uint32_t G, uint32_t b, uint32_t w, uint32_t nw) {
    CSmem s;
    const uint32_t tile = G * b * w;
    const uint32_t rec = record_max_bytes(G, b, w);
    s.buf_bytes = ((tile > rec ? tile : rec) + 16 + 15) & ~15u;
    s.buf_stride = (s.buf_bytes + 1023) & ~1023u;
    // one metadata block per stage
    uint32_t m = 0;
    auto mtake = [&](uint32_t bytes) {
        m = (m + 15) & ~15u;
        const uint32_t at = m;
        m += bytes;
        return at;
    };
    s.m_kind = mtake(G);
    s.m_w = mtake(16 * nw);
    s.meta_stride = (m + 15) & ~15u;
    s.meta0 = (kStages - 1) * s.buf_stride + s.buf_bytes;  // after the last buffer (16-aligned)
    s.lut = s.meta0 + kStages * s.meta_stride;
    uint32_t o = s.lut + 256 * 16;
    // f64: the tile's block statistics exchange, 16 bytes a block
    s.xs = 0;
    if (w == 8) {
        s.xs = (o + 15) & ~15u;
        o = s.xs + 16 * G;
    }
    s.total = ((o + 1023) & ~1023u) + 1024;  // + slack to realign the dynamic base
    return s;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------

template <typename T, int LPB, int VPL, int NW, bool BATCH>
__global__ void __launch_bounds__(compress_threads(NW),
                                  (tile_blocks(LPB * VPL, sizeof(T)) * LPB * VPL * sizeof(T) > 32768) ? 1 : 2)
    compress_kernel(const __grid_constant__ CField one, const __grid_constant__ CompressLaunch lc) {
    using F = Fmt<T>;
    using U = typename F::U;
    constexpr int w = F::w;
    constexpr int W = F::W;
    constexpr int kConsumerWarps = NW;
    constexpr int kCThreads = compress_threads(NW);
    constexpr int kProducerWarp = NW;
    constexpr int kStorerWarp = NW + 1;
    constexpr int BPW = 32 / LPB;       // blocks per warp
    constexpr int RPL = VPL * w / 128;  // 128-byte rows per lane
    constexpr int NCODE = (2 * VPL + 31) / 32;
    static_assert(RPL >= 1 && NCODE >= 1, "lane geometry");

    extern __shared__ __align__(16) uint8_t smem_raw[];  // realigned to 1024 below
    // full: tile copied in; encoded: every consumer warp has its blocks'
    // totals in place; ready: record written; empty: record stored
    __shared__ __align__(8) uint64_t full[kStages], encoded[kStages], ready[kStages], empty[kStages];
    // f64 (XS): the warps' block keys are in the exchange table; the block
    // statistics are in it (per tile, in tile order)
    __shared__ __align__(8) uint64_t keys_in, stats_out;
    // per stage: the field and its local tile (0xFFFFFFFF: no more tiles)
    __shared__ uint32_t st_field[kStages], st_tile[kStages], st_rec[kStages];

    // the 128-byte swizzle of the tensor copy needs 1024-byte aligned buffers
    uint8_t *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    constexpr uint32_t b = (uint32_t)(LPB * VPL);
    constexpr uint32_t G = tile_blocks(b, (uint32_t)w);
    constexpr uint32_t TILE_ROWS = G * b * w / 128;  // 256, or 512 for 64 KiB tiles
    constexpr uint32_t TILE_BOXES = TILE_ROWS / 256;  // tensor copies of 256 rows
    static_assert((uint32_t)(NW * 32 * RPL) == TILE_ROWS, "the tile is laid out over the consumers' lanes");
    const CSmem L = compress_smem(G, b, w, NW);
    uint32_t *lut = reinterpret_cast<uint32_t *>(smem + L.lut);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(kPlaneLut.v);
        uint4 *dst = reinterpret_cast<uint4 *>(lut);
        for (int i = tid; i < 256; i += kCThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&encoded[i], kConsumerWarps);
            mbar_init(&ready[i], kConsumerWarps);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&keys_in, kConsumerWarps);
        mbar_init(&stats_out, 1);
        fence_mbar_init();
        for (int i = 0; i < kStages; ++i) {
            st_tile[i] = 0xFFFFFFFFu;
            st_field[i] = 0;
            st_rec[i] = 0;
        }
    }
    __syncthreads();
    // nothing above reads or writes memory that an earlier kernel may write
    // (the launch may be the programmatic dependent of the workspace clear)
    wait_prior_grids();

    if (warp == kProducerWarp) {
        // ---- producer: tickets and tile copies into the stage ring ---------
        if (lane != 0) return;
        // per stage: is the last phase a copy (then it may still be in flight
        // when the producer is done), and its phase index
        uint32_t copy_last = 0, copy_par = 0;  // bit st
        for (uint32_t it = 0;; ++it) {
            const int st = (int)(it % kStages);
            const uint32_t k = it / kStages;
            if (it >= kStages && !mbar_wait_bounded(&empty[st], (k - 1) & 1u, lc.lookback_ns + lc.copy_ns)) {
                atomicOr(lc.err, kErrTimeout);
                break;
            }
            // Take tile it's ticket only once the warps have finished tile
            // it - 2 (they are on tile it - 1 now): a ticket taken earlier
            // would wait in the ring longer, the tiles before it in ticket
            // order would be encoded later, and so the look-back -- which
            // holds a stage until every earlier tile has its aggregate --
            // would wait longer.  The copy still has a tile's time to land.
            if (it >= 2) {
                const uint32_t j = it - 2;
                if (!mbar_wait_bounded(&ready[j % kStages], (j / kStages) & 1u, lc.lookback_ns + lc.copy_ns)) {
                    atomicOr(lc.err, kErrTimeout);
                    break;
                }
            }
            // a ticket is a tile of the launch's global list; find its field
            const uint64_t t = atomicAdd(lc.ticket, 1u);
            const bool more = t < lc.total_tiles;
            const uint32_t f = more ? field_of<BATCH>(lc, t) : 0u;
            const CField *F = field_ptr<BATCH>(one, lc, f);
            const uint32_t tile = more ? (uint32_t)(t - F->tile0) : 0xFFFFFFFFu;
            st_field[st] = f;
            st_tile[st] = tile;
            const uint64_t row0 = (uint64_t)tile * TILE_ROWS;
            if (more && F->use_tma && row0 < F->rows_full) {
                mbar_arrive_expect_tx(&full[st], TILE_ROWS * 128u);
                // the input is read once: its lines go first when L2 needs room,
                // before other kernels' lines still waiting to be written back
                uint64_t pol;
                asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#pragma unroll
                for (int i = 0; i < (int)TILE_BOXES; ++i) {
                    const uint32_t dst = smem_addr(smem + st * L.buf_stride + i * 32768);
                    const int y = (int)(row0 + 256 * i);
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
                        "[%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
                        "l"(reinterpret_cast<uint64_t>(&F->tmap)), "r"(0), "r"(y), "r"(smem_addr(&full[st])), "l"(pol)
                        : "memory");
                }
                copy_last |= 1u << st;
                copy_par = (copy_par & ~(1u << st)) | ((k & 1u) << st);
            } else {
                // a later phase on this stage implies its earlier copy was consumed
                mbar_arrive(&full[st]);
                copy_last &= ~(1u << st);
            }
            if (!more) break;
        }
        // do not leave while a copy may still be writing into shared memory
        for (int st = 0; st < kStages; ++st)
            if ((copy_last >> st) & 1u) mbar_wait_bounded(&full[st], (copy_par >> st) & 1u, lc.copy_ns);
        return;
    }

    if (warp == kStorerWarp) {
        // ---- storer: look-back, index entry, record store --------------------
        for (uint32_t it = 0;; ++it) {
            const int st = (int)(it % kStages);
            const uint32_t k = it / kStages;
            if (!mbar_wait_bounded(&ready[st], k & 1u, lc.lookback_ns + 4 * lc.copy_ns)) {
                if (lane == 0) atomicOr(lc.err, kErrTimeout);
                break;
            }
            const uint32_t tile = st_tile[st];
            if (tile == 0xFFFFFFFFu) break;
            const CField *F = field_ptr<BATCH>(one, lc, st_field[st]);
            const Geometry &g = F->g;
            uint64_t *lookback = F->lookback;
            const uint32_t rec_bytes = st_rec[st];
            auto counts_and_state = [&]() {
                // the field's counts (the header is written once every CTA is
                // done) and the tile's state bits, from the warps' totals and
                // the block kinds in the stage's metadata
                const uint8_t *meta = smem + (L.meta0 + st * L.meta_stride);
                const uint4 wt = lane < kConsumerWarps ? reinterpret_cast<const uint4 *>(meta + L.m_w)[lane]
                                                       : make_uint4(0, 0, 0, 0);
                const uint32_t nn_t = __reduce_add_sync(kFull, wt.x) >> 20;
                const uint32_t raw_t = __reduce_add_sync(kFull, wt.y), esc_t = __reduce_add_sync(kFull, wt.z);
                if (lane == 0) {
                    Workspace *ws = F->ws;
                    if (nn_t) atomicAdd(&ws->nn, (unsigned long long)nn_t);
                    if (raw_t) atomicAdd(&ws->nraw, (unsigned long long)raw_t);
                    if (esc_t) atomicAdd(&ws->nesc, (unsigned long long)esc_t);
                }
                // bit i of byte j is set when block 8j + i is not constant
                const uint8_t *sm_kind = meta + L.m_kind;
                const uint64_t k0 = (uint64_t)tile * G;
                const uint32_t Gt = (uint32_t)min_u64(G, g.nb - k0);
                uint8_t *state = F->out + g.off_state + (size_t)k0 / 8;
                for (uint32_t j = lane; j < (Gt + 7) / 8; j += 32) {
                    uint32_t byte = 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint32_t kk = j * 8 + i;
                        if (kk < Gt && sm_kind[kk] != kConst) byte |= 1u << i;
                    }
                    state[j] = (uint8_t)byte;
                }
            };
            // A tile whose record is empty (every block constant) has nothing
            // to store: its counts and state bits go out now, and its buffer
            // is free before the look-back.  Otherwise they go out while the
            // store reads the record.
            const bool empty_rec = rec_bytes == 0;
            if (empty_rec) {
                counts_and_state();
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
            }
            // warp-parallel decoupled look-back: 32 predecessors per probe,
            // lane i looking at tile - 1 - i; stop at the nearest inclusive
            // prefix, adding the aggregates in between
            uint64_t excl = 0;
            bool timed_out = false;
            {
                const uint64_t t0 = globaltimer_ns();
                int64_t base = (int64_t)tile - 1;
                while (base >= 0) {
                    const int64_t j = base - lane;
                    const uint64_t wv = j >= 0 ? ld_relaxed_u64(&lookback[j]) : kFlagPrefix;
                    const uint64_t flag = wv & ~kValueMask;
                    const uint32_t pre = __ballot_sync(kFull, flag == kFlagPrefix);
                    const uint32_t inv = __ballot_sync(kFull, flag == 0);
                    const int first_p = pre ? __ffs(pre) - 1 : 32;
                    const uint32_t need = first_p >= 31 ? kFull : ((2u << first_p) - 1u);
                    if (inv & need) {
                        // one lane's clock decides, so the warp stays converged
                        if (__shfl_sync(kFull, (int)(globaltimer_ns() - t0 > lc.lookback_ns), 0)) {
                            timed_out = true;
                            break;
                        }
                        __nanosleep(256);  // a predecessor is still encoding
                        continue;
                    }
                    uint64_t v = lane <= first_p ? (wv & kValueMask) : 0ull;
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
                    excl += v;
                    if (first_p < 32) break;
                    base -= 32;
                }
            }
            uint8_t *out = F->out;
            if (lane == 0) {
                st_relaxed_u64(&lookback[tile], kFlagPrefix | (excl + rec_bytes));
                Workspace *ws = F->ws;
                if (timed_out) {
                    atomicOr(&ws->err, kErrTimeout);
                    atomicAdd(&ws->lookback_timeouts, 1ull);
                    atomicCAS(&ws->first_lb_tile, 0u, tile + 1);
                }
                uint64_t *idx = reinterpret_cast<uint64_t *>(out + g.off_index);
                idx[tile] = excl;
                if (tile == g.ntiles - 1) {
                    idx[g.ntiles] = excl + rec_bytes;
                    const uint64_t state_end = g.off_state + (g.nb + 7) / 8;
                    for (uint64_t i = state_end; i < g.off_mu; ++i) out[i] = 0;
                    for (uint64_t i = g.off_mu + g.nb * w; i < g.off_index; ++i) out[i] = 0;
                    for (uint64_t i = g.off_index + 8 * (g.ntiles + 1); i < g.off_rec; ++i) out[i] = 0;
                }
                if (rec_bytes) {
                    fence_proxy_async_smem();
                    bulk_s2g(out + g.off_rec + excl, smem + st * L.buf_stride, rec_bytes);
                    bulk_commit();
                }
            }
            if (!empty_rec) {
                counts_and_state();
                __syncwarp();
                if (lane == 0) {
                    // the buffer is free once the store has read it
                    bulk_wait_read_all();
                    mbar_arrive(&empty[st]);
                }
            }
            __syncwarp();
        }
        // the last CTA to get here writes every field's header and result
        uint32_t last = 0;
        if (lane == 0) {
            __threadfence();
            last = atomicAdd(lc.done, 1u) == gridDim.x - 1 ? 1u : 0u;
            if (last) __threadfence();
        }
        last = __shfl_sync(kFull, last, 0);
        if (last) {
            const uint32_t launch_err = *reinterpret_cast<volatile uint32_t *>(lc.err);
            for (uint32_t f = lane; f < lc.nfields; f += 32) {
                const CField *F = field_ptr<BATCH>(one, lc, f);
                const Geometry &g = F->g;
                volatile Workspace *ws = F->ws;
                const uint64_t rec_total = reinterpret_cast<volatile uint64_t *>(F->out + g.off_index)[g.ntiles];
                const uint64_t total = g.off_rec + rec_total;
                uint32_t *h32 = reinterpret_cast<uint32_t *>(F->out);
                uint64_t *h64 = reinterpret_cast<uint64_t *>(F->out);
                h32[0] = kMagic;
                h32[1] = kVersion | (F->dtype << 8);
                h32[2] = b;
                h32[3] = G;
                h64[2] = g.n;
                h64[3] = F->e_bits;
                h64[4] = ws->nn;
                h64[5] = ws->nraw;
                h64[6] = ws->nesc;
                h64[7] = total;
                const uint32_t err = ws->err | launch_err;
                const uint64_t status = (err & (kErrTimeout | kErrTmaTimeout)) ? 6ull
                                        : (err & kErrInternal)                 ? 5ull
                                                                               : 0ull;
                ws->result[0] = total;
                ws->result[1] = status;
                if (F->d_result) {
                    F->d_result[0] = total;
                    F->d_result[1] = status;
                }
            }
        }
        return;
    }

    // ---- consumers (warps 0..7): encode tiles into records ------------------
    // The warps of a CTA meet once per tile (the `encoded` mbarrier, after
    // which the tile's totals are known); every wait is bounded.
    for (uint32_t it = 0;; ++it) {
        const int st = (int)(it % kStages);
        const uint32_t k = it / kStages;
        const bool waited = mbar_wait_bounded(&full[st], k & 1u, lc.copy_ns);
        const uint32_t tile = waited ? st_tile[st] : 0xFFFFFFFFu;
        if (tile == 0xFFFFFFFFu) {
            // the producer is done (or the copy never arrived): hand the stage
            // to the storer, which stops on it, and stop
            if (!waited && lane == 0) {
                atomicOr(lc.err, kErrTmaTimeout);
                st_tile[st] = 0xFFFFFFFFu;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[st]);
            break;
        }
        const CField *Fd = field_ptr<BATCH>(one, lc, st_field[st]);
        const Geometry &g = Fd->g;
        const T e = F::from((U)Fd->e_bits);
        uint8_t *buf = smem + st * L.buf_stride;
        uint8_t *meta = smem + (L.meta0 + st * L.meta_stride);
        uint8_t *sm_kind = meta + L.m_kind;
        uint4 *sm_w = reinterpret_cast<uint4 *>(meta + L.m_w);  // per warp: nn << 20 | mid, raw, escalated
        const uint64_t k0 = (uint64_t)tile * G;
        const uint32_t Gt = (uint32_t)min_u64(G, g.nb - k0);
        const uint64_t row0 = (uint64_t)tile * TILE_ROWS;
        const uint64_t rows_full = Fd->rows_full;
        const bool tma = Fd->use_tma && row0 < rows_full;

        // Tiles wholly inside the input (all but its ragged end) run a copy of
        // the work below compiled with every block full and every row copied
        // in: no checks of the input's end per block, row or group of values
        const bool full_tile = tma && (k0 + G) * b <= g.n;
        auto tile_body = [&](auto full_c) -> bool {
            constexpr bool FT = decltype(full_c)::value;
            // ---- 1. block statistics and encoding (registers) -------------------
            const int sub = lane % LPB;
            const uint32_t blk = (uint32_t)(warp * BPW + lane / LPB);
            const bool exists = FT || blk < Gt;
            const uint64_t kg = k0 + blk;
            const int len = FT ? (int)b : (exists ? (int)min_u64(b, g.n - kg * b) : 0);
            int nvalid = VPL;
            if constexpr (!FT) {
                nvalid = len - sub * VPL;
                nvalid = nvalid < 0 ? 0 : (nvalid > VPL ? VPL : nvalid);
            }
            const bool full_lane = FT || nvalid == VPL;
            const uint32_t lane_row0 = (uint32_t)((warp * 32 + lane) * RPL);
            // the lane's values in global memory (read only below nvalid)
            const U *src = reinterpret_cast<const U *>(Fd->in) + kg * b + sub * VPL;

            // rows the tensor copy brought in come from shared memory; the
            // input's ragged end (or every row without the tensor copy) from global
            constexpr int VPR = 128 / w;  // values per row
            U x[VPL];
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr) {
                const uint32_t rowi = lane_row0 + rr;
                if (FT || (tma && row0 + rowi < rows_full)) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(buf + (rowi << 7) + ((c ^ (rowi & 7u)) << 4));
                        const U *u = reinterpret_cast<const U *>(&v);
#pragma unroll
                        for (int kk = 0; kk < 16 / w; ++kk) x[rr * VPR + c * (16 / w) + kk] = u[kk];
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < VPR; ++m) x[rr * VPR + m] = rr * VPR + m < nvalid ? src[rr * VPR + m] : U(0);
                }
            }
            // this lane's rows are read: clear them, the buffer becomes the record
            // (the exact slow path below re-reads the input from global memory)
            {
                const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) {
                    const uint32_t rowi = lane_row0 + rr;
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        *reinterpret_cast<uint4 *>(buf + (rowi << 7) + ((c ^ (rowi & 7u)) << 4)) = z;
                }
                if (warp == kConsumerWarps - 1)
                    for (uint32_t i = TILE_ROWS * 128u + 16u * lane; i < L.buf_bytes; i += 16u * 32u)
                        *reinterpret_cast<uint4 *>(buf + i) = z;
            }
            uint32_t codes[NCODE];
            int kind, req, req0;
            T mu;
            uint32_t mk_lane;
            // f64 with 128 <= b <= 512, one field: the block statistics of the
            // whole tile on warp 0, in one pass over its blocks (an FP64
            // instruction costs a warp's issue whatever lanes it runs on, and a
            // warp holds only 4 blocks or fewer); the other warps wait for
            // them.  At b = 64 warp 0 needs two passes, at b = 1024 (one CTA
            // per SM) nothing hides the wait, and the batch instances spill
            // registers with it: all three are slower that way.
            constexpr bool XS = !BATCH && sizeof(T) == 8 && LPB * VPL >= 128 && LPB * VPL <= 512;
            const uint32_t xpar = it & 1u;  // the exchange barriers' phase: one per tile
            auto xchg = [&](typename F::S kmn, typename F::S kmx, XOut<T> &o) -> bool {
                longlong2 *xt = reinterpret_cast<longlong2 *>(smem + L.xs);
                if (exists && sub == 0) xt[blk] = make_longlong2((long long)kmn, (long long)kmx);
                __syncwarp();
                if (lane == 0) mbar_arrive(&keys_in);
                if (warp == 0) {
                    if (!mbar_wait_bounded(&keys_in, xpar, lc.copy_ns)) return false;
                    for (uint32_t i = (uint32_t)lane; i < G; i += 32) {
                        const longlong2 v = xt[i];
                        const BlockStats<T> bs =
                            block_stats<T>((typename F::S)v.x, (typename F::S)v.y, FT || i < Gt, e);
                        const bool chk = bs.kind == kNonConst &&
                                         bound_check_needed<T>(bs.mn, bs.mx, bs.mu, bs.R, (U)Fd->e_bits);
                        xt[i] = make_longlong2((long long)F::bits(bs.mu),
                                               (long long)((uint32_t)bs.kind | ((uint32_t)bs.req0 << 8) |
                                                           ((uint32_t)chk << 16)));
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&stats_out);
                }
                if (!mbar_wait_bounded(&stats_out, xpar, lc.copy_ns)) return false;
                const longlong2 v = xt[blk];
                const uint32_t m = (uint32_t)v.y;
                o.mu = F::from((U)v.x);
                o.kind = exists ? (int)(m & 0xFFu) : 0xFF;
                o.req0 = (int)((m >> 8) & 0xFFu);
                o.check = ((m >> 16) & 1u) != 0u;
                return true;
            };
            bool encoded_ok;
            if (FT || __all_sync(kFull, full_lane)) {
                encoded_ok = encode_lane<T, LPB, VPL, true, XS>(x, codes, kind, req, req0, mu, mk_lane, src, nvalid,
                                                                exists, e, Fd->e_bits, Fd->ws, tile, xchg);
            } else {
                encoded_ok = encode_lane<T, LPB, VPL, false, XS>(x, codes, kind, req, req0, mu, mk_lane, src,
                                                                 nvalid, exists, e, Fd->e_bits, Fd->ws, tile, xchg);
            }
            if (!encoded_ok) {
                // the statistics exchange ran out of time: give up on the tile
                if (lane == 0) {
                    atomicOr(lc.err, kErrTimeout);
                    st_tile[st] = 0xFFFFFFFFu;
                    mbar_arrive(&ready[st]);
                }
                return false;
            }
            const bool lead = exists && sub == 0;  // the block's first lane
            if (lead) {
                sm_kind[blk] = (uint8_t)kind;
                reinterpret_cast<U *>(Fd->out + g.off_mu)[kg] = kind == kRaw ? U(0) : F::bits(mu);
            }
            // the warp's totals; its blocks are consecutive, so an exclusive scan
            // over lanes gives each block's mid-byte offset inside the warp's share
            uint32_t mid_w;
            const uint32_t lane_excl = warp_exclusive_scan(mk_lane, &mid_w);
            const uint32_t nonc_bal = __ballot_sync(kFull, lead && kind != kConst);
            const uint32_t raw_bal = __ballot_sync(kFull, lead && kind == kRaw);
            const uint32_t esc_bal = __ballot_sync(kFull, lead && kind == kNonConst && req > req0);
            // per warp: (non-constant blocks << 20 | mid bytes), raw blocks, escalated blocks
            if (lane == 0)
                sm_w[warp] = make_uint4((uint32_t)__popc(nonc_bal) << 20 | mid_w, __popc(raw_bal), __popc(esc_bal), 0);
            __syncwarp();
            if (lane == 0) mbar_arrive(&encoded[st]);

            // per-lane counts of values with code <= j (j = 0, 1, 2), packed in
            // FB-bit fields, and their exclusive scan over the block's lanes;
            // nothing here depends on the other warps, so it runs before the wait.
            // Every lane runs this (the shuffles need the whole warp); lanes of
            // constant or raw blocks contribute nothing.
            const uint32_t mk_blk_excl = __shfl_sync(kFull, lane_excl, lane & ~(LPB - 1));
            const uint32_t rank_in_warp = __popc(nonc_bal & ((1u << (lane & ~(LPB - 1))) - 1u));
            using CntT = std::conditional_t<(LPB * VPL > 1023), unsigned long long, uint32_t>;
            constexpr int FB = LPB * VPL > 1023 ? 16 : 10;
            constexpr CntT FM = (CntT(1) << FB) - 1;
            CntT cnt = 0;
            if (exists && kind == kNonConst) {
#pragma unroll
                for (int i = 0; i < NCODE; ++i) {
                    const int nv = nvalid - 16 * i;
                    const uint32_t vm = nv >= 16 ? 0x55555555u : (nv <= 0 ? 0u : (0x55555555u >> (2 * (16 - nv))));
                    const uint32_t lo = codes[i] & 0x55555555u, hi = (codes[i] >> 1) & 0x55555555u;
                    cnt += (CntT)__popc(~(lo | hi) & vm) | ((CntT)__popc(~hi & vm) << FB) |
                           ((CntT)__popc(~(lo & hi) & vm) << (2 * FB));
                }
            }
            CntT incl = cnt;
#pragma unroll
            for (int d = 1; d < LPB; d <<= 1) {
                const CntT y = __shfl_up_sync(kFull, incl, d);
                if (sub >= d) incl += y;
            }
            const CntT tot = __shfl_sync(kFull, incl, (lane & ~(LPB - 1)) + LPB - 1);
            const CntT off = incl - cnt;

            if (!mbar_wait_bounded(&encoded[st], k & 1u, lc.lookback_ns + lc.copy_ns)) {
                // a warp of this CTA never finished the tile: give up
                if (lane == 0) {
                    atomicOr(lc.err, kErrTimeout);
                    st_tile[st] = 0xFFFFFFFFu;
                    mbar_arrive(&ready[st]);
                }
                return false;
            }

            // ---- 2. tile totals and the aggregate for the look-back --------------
            // lane i holds warp i's (nn << 20 | mid); warp reductions give the
            // tile's totals and the sums over the warps before this one
            const uint32_t wt = lane < kConsumerWarps ? sm_w[lane].x : 0u;
            const uint32_t nm_t = __reduce_add_sync(kFull, wt);
            const uint32_t nm_before = __reduce_add_sync(kFull, lane < warp ? wt : 0u);
            const uint32_t nn_t = nm_t >> 20, mid_t = nm_t & 0xFFFFFu;
            const uint32_t nn_before = nm_before >> 20, mid_before = nm_before & 0xFFFFFu;
            const uint32_t rec_bytes = (uint32_t)pad16((uint64_t)nn_t * (b / 4 + 1) + mid_t);
            if (warp == 0 && lane == 0) {
                st_rec[st] = rec_bytes;
                st_relaxed_u64(&Fd->lookback[tile], kFlagAgg | rec_bytes);
            }
            if (SZX_CHECKS && rec_bytes > record_max_bytes(G, b, w) && tid == 0) report_bad(Fd->ws, tile, 2);
            const uint32_t rank = nn_before + rank_in_warp;

            // ---- 3. the record --------------------------------------------------
            uint32_t *words = reinterpret_cast<uint32_t *>(buf);
            // every record write goes through put() (positions in bits, c8 = 8 x
            // bytes): a self-checked build verifies that it lands inside the record
            auto put = [&](uint32_t pb, uint32_t run, uint32_t c8) {
                // (a run of no bytes -- a group past a partial block's end -- ORs
                // zeros: only its words must lie in the buffer)
                if (SZX_CHECKS && ((pb >> 3) + 8 > L.buf_bytes || (c8 && ((pb + c8) >> 3) > rec_bytes))) {
                    report_bad(Fd->ws, tile, 1);
                    return;
                }
                or_bytes(words, pb, run);
            };
            // whole words of a dense plane-2 run: OR for the two edge words
            // (shared with the writers before and after), a plain store for a
            // word this lane alone writes
            auto or_word = [&](uint32_t widx, uint32_t v) {
                if (SZX_CHECKS && 4 * widx + 4 > L.buf_bytes) {
                    report_bad(Fd->ws, tile, 4);
                    return;
                }
                atomicOr(words + widx, v);
            };
            auto put_word = [&](uint32_t widx, uint32_t v) {
                if (SZX_CHECKS && 4 * widx + 4 > rec_bytes) {
                    report_bad(Fd->ws, tile, 5);
                    return;
                }
                words[widx] = v;
            };
            // Does every plane-2 run of the warp hold byte 2 of all its lane's
            // values (no code 3, every value valid)?  Then each word of such a
            // run is one funnel shift of two consecutive 4-byte groups (see
            // below).  Decided for the whole warp, so that no lane diverges.
            bool dense2;
            {
                const int s2 = (8 - (req & 7)) & 7;
                const bool has2 = exists && kind == kNonConst && ((req + s2) >> 3) >= 3;
                const bool all2 = full_lane && (uint32_t)((cnt >> (2 * FB)) & FM) == (uint32_t)VPL;
                dense2 = __all_sync(kFull, !has2 || all2);
            }
            if (exists && kind != kConst) {
                const uint32_t mbase = nn_t * (b / 4 + 1) + mid_before + mk_blk_excl;
                if (sub == 0) {
                    // the reqBits byte's word may also hold mid bytes: OR it in too
                    const uint32_t p = nn_t * (b / 4) + rank;
                    atomicOr(words + (p >> 2), (kind == kNonConst ? (uint32_t)req : 0xFFu) << (8 * (p & 3u)));
                }
                if (kind == kRaw) {
                    // verbatim input bytes, value-major
                    const U *src = reinterpret_cast<const U *>(Fd->in) + kg * b + sub * VPL;
                    for (int m = 0; m < nvalid; ++m) {
                        const U v = src[m];
                        const uint32_t p = mbase + (uint32_t)(sub * VPL + m) * w;
#pragma unroll
                        for (int h = 0; h < w / 4; ++h) put(8 * (p + 4 * h), (uint32_t)(v >> (32 * h)), 32);
                    }
                } else {
                    // lead codes: this lane's values are bytes [sub*VPL/4, (sub+1)*VPL/4)
                    if (SZX_CHECKS && (rank + 1) * (b / 4) > nn_t * (b / 4)) report_bad(Fd->ws, tile, 6);
                    uint8_t *lead = buf + rank * (b / 4) + sub * (VPL / 4);
                    if constexpr (NCODE == 4) {
                        *reinterpret_cast<uint4 *>(lead) = make_uint4(codes[0], codes[1], codes[2], codes[3]);
                    } else if constexpr (NCODE == 2) {
                        *reinterpret_cast<uint2 *>(lead) = make_uint2(codes[0], codes[1]);
                    } else {
                        *reinterpret_cast<uint32_t *>(lead) = codes[0];
                    }
                    const int s = (8 - (req & 7)) & 7;
                    const int q = (req + s) >> 3;
                    const uint32_t n0 = (uint32_t)(tot & FM), n1 = (uint32_t)((tot >> FB) & FM),
                                   n2 = (uint32_t)((tot >> (2 * FB)) & FM);
                    // plane positions in bits
                    uint32_t pos0 = 8 * (mbase + (uint32_t)(off & FM));
                    uint32_t pos1 = 8 * (mbase + n0 + (uint32_t)((off >> FB) & FM));
                    uint32_t pos2 = 8 * (mbase + n0 + n1 + (uint32_t)((off >> (2 * FB)) & FM));
                    const uint32_t dense0 = mbase + n0 + n1 + n2 + (uint32_t)sub * VPL;
                    uint32_t w2prev = 0;  // plane 2 on the dense path: the previous group's bytes
#pragma unroll
                    for (int gq = 0; gq < VPL / 4; ++gq) {
                        // lookup codes: values past the end of a partial block never match
                        uint32_t code8 = (codes[gq >> 2] >> (8 * (gq & 3))) & 0xFFu;
                        uint32_t dense8 = 0;
                        if (!full_lane) {
                            const int nv = nvalid - 4 * gq;
                            const uint32_t inval = nv >= 4 ? 0u : (nv <= 0 ? 0xFFu : (0xFFu << (2 * nv)) & 0xFFu);
                            code8 |= inval;
                            dense8 = inval;
                        }
                        uint32_t Wd[W / 8];
                        if constexpr (sizeof(T) == 4) {
                            uint32_t Wq[4];
                            transpose4((uint32_t)x[4 * gq], (uint32_t)x[4 * gq + 1], (uint32_t)x[4 * gq + 2],
                                       (uint32_t)x[4 * gq + 3], Wq);
#pragma unroll
                            for (int j = 0; j < 4; ++j) Wd[j] = Wq[j];
                        } else {
                            uint32_t Wh[4], Wl[4];
                            transpose4((uint32_t)(x[4 * gq] >> 32), (uint32_t)(x[4 * gq + 1] >> 32),
                                       (uint32_t)(x[4 * gq + 2] >> 32), (uint32_t)(x[4 * gq + 3] >> 32), Wh);
                            transpose4((uint32_t)x[4 * gq], (uint32_t)x[4 * gq + 1], (uint32_t)x[4 * gq + 2],
                                       (uint32_t)x[4 * gq + 3], Wl);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                Wd[j] = Wh[j];
                                Wd[4 + j] = Wl[j];
                            }
                        }
                        const uint4 e = reinterpret_cast<const uint4 *>(lut)[code8];
                        put(pos0, prmt(Wd[0], 0, e.x), e.x >> 16);
                        pos0 += e.x >> 16;
                        put(pos1, prmt(Wd[1], 0, e.y), e.y >> 16);
                        pos1 += e.y >> 16;
                        if (q >= 3) {
                            if (dense2) {
                                // word gq of the run holds the tail of group
                                // gq - 1 and the head of group gq; only the
                                // first word is shared with the writer before
                                // it (OR), the others are this lane's alone
                                if (gq == 0) or_word(pos2 >> 5, __funnelshift_l(0u, Wd[2], pos2));
                                else put_word((pos2 >> 5) + gq, __funnelshift_l(w2prev, Wd[2], pos2));
                                w2prev = Wd[2];
                            } else {
                                put(pos2, prmt(Wd[2], 0, e.z), e.z >> 16);
                                pos2 += e.z >> 16;
                            }
                        }
                        if (q >= 4) {
                            const uint32_t sel = full_lane ? (0x3210u | (32u << 16)) : lut[4 * dense8 + 2];
#pragma unroll
                            for (int j = 3; j < W / 8; ++j) {
                                if (j < q)
                                    put(8 * (dense0 + (uint32_t)(j - 3) * len + 4 * gq), prmt(Wd[j], 0, sel),
                                        sel >> 16);
                            }
                        }
                    }
                    // the dense run's last word is shared with the writer after it
                    if (dense2 && q >= 3) or_word((pos2 >> 5) + VPL / 4, __funnelshift_l(w2prev, 0u, pos2));
                }
            }
            // hand the record to the storer (its bulk store reads it through the
            // async proxy)
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[st]);
            return true;
        };
        if (!(full_tile ? tile_body(std::true_type{}) : tile_body(std::false_type{}))) break;
    }
}


__global__ void clear_words_kernel(uint32_t *p, uint64_t n) {
    // the kernel behind this one may start now (it waits for this one to end
    // before its first global access)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = 0u;
}

// ---------------------------------------------------------------------------
// host side

cudaError_t launch_clear_words(uint32_t *p, uint64_t n, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const uint64_t ctas = min_u64((n + 255) / 256, 4 * 148);
    clear_words_kernel<<<(unsigned)ctas, 256, 0, stream>>>(p, n);
    return cudaGetLastError();
}

namespace {

template <typename T, int LPB, int VPL, int NW>
cudaError_t launch_t(const CField &one, const CompressLaunch &lc, int ctas_per_sm, bool pdl, cudaStream_t stream) {
    constexpr uint32_t b = (uint32_t)(LPB * VPL), w = (uint32_t)Fmt<T>::w;
    const CSmem L = compress_smem(tile_blocks(b, w), b, w, NW);
    auto kern = lc.fields ? compress_kernel<T, LPB, VPL, NW, true> : compress_kernel<T, LPB, VPL, NW, false>;
    // per device and kernel: the shared-memory attribute and the occupancy,
    // set up on first use (a launch then only reads them)
    int per_sm = 0, sms = 0;
    cudaError_t err =
        launch_setup(reinterpret_cast<const void *>(kern), L.total, compress_threads(NW), &per_sm, &sms);
    if (err != cudaSuccess) return err;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    const uint64_t grid = min_u64(lc.total_tiles, (uint64_t)sms * per_sm);
    return launch_kernel(kern, (unsigned)grid, compress_threads(NW), L.total, pdl, stream, one, lc);
}

// The kernel instance for (dtype, block, consumer warps): 8 warps with 32
// values per lane (16 for f64), or 4 warps with twice as many values per lane
// where a block still covers whole lanes (not for f32 with b = 32, nor f64
// with b = 1024, whose 64 values per lane would not fit the registers).
cudaError_t dispatch(int dtype, uint32_t block, int nw, const CField &one, const CompressLaunch &lc,
                     int ctas_per_sm, bool pdl, cudaStream_t stream) {
    if (nw == 0) nw = 8;
    if (dtype == 0 && nw == 8) {
        switch (block) {
            case 32: return launch_t<float, 1, 32, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 64: return launch_t<float, 2, 32, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 128: return launch_t<float, 4, 32, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 256: return launch_t<float, 8, 32, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 512: return launch_t<float, 16, 32, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 1024: return launch_t<float, 32, 32, 8>(one, lc, ctas_per_sm, pdl, stream);
        }
    } else if (dtype == 0 && nw == 4) {
        switch (block) {
            case 64: return launch_t<float, 1, 64, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 128: return launch_t<float, 2, 64, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 256: return launch_t<float, 4, 64, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 512: return launch_t<float, 8, 64, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 1024: return launch_t<float, 16, 64, 4>(one, lc, ctas_per_sm, pdl, stream);
        }
    } else if (dtype == 1 && nw == 8) {
        switch (block) {
            case 32: return launch_t<double, 2, 16, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 64: return launch_t<double, 4, 16, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 128: return launch_t<double, 8, 16, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 256: return launch_t<double, 16, 16, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 512: return launch_t<double, 32, 16, 8>(one, lc, ctas_per_sm, pdl, stream);
            case 1024: return launch_t<double, 32, 32, 8>(one, lc, ctas_per_sm, pdl, stream);
        }
    } else if (dtype == 1 && nw == 4) {
        switch (block) {
            case 32: return launch_t<double, 1, 32, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 64: return launch_t<double, 2, 32, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 128: return launch_t<double, 4, 32, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 256: return launch_t<double, 8, 32, 4>(one, lc, ctas_per_sm, pdl, stream);
            case 512: return launch_t<double, 16, 32, 4>(one, lc, ctas_per_sm, pdl, stream);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_compress(const void *in, uint64_t n, int dtype, uint64_t e_bits, uint32_t block,
                            void *out, uint64_t ws_offset, uint64_t *d_result, cudaStream_t stream, Clear clear) {
    return launch_compress_ws(in, n, dtype, e_bits, block, out, static_cast<uint8_t *>(out) + ws_offset,
                              d_result, stream, clear);
}

void fill_compress_field(CField *f, const void *in, uint64_t n, int dtype, uint64_t e_bits, uint32_t block,
                         void *out, void *ws, uint64_t *d_result, uint64_t tile0) {
    CField &c = *f;
    std::memset(&c, 0, sizeof(c));
    const uint32_t w = dtype == 0 ? 4 : 8;
    c.in = static_cast<const uint8_t *>(in);
    c.out = static_cast<uint8_t *>(out);
    c.g = make_geometry(n, block, w);
    c.ws = reinterpret_cast<Workspace *>(ws);
    c.lookback = reinterpret_cast<uint64_t *>(static_cast<uint8_t *>(ws) + kWsHeader);
    c.d_result = d_result;
    c.e_bits = e_bits;
    c.dtype = (uint32_t)dtype;
    c.rows_full = n * w / 128;
    c.tile0 = tile0;
    c.use_tma = encode_row_map(&c.tmap, in, c.rows_full, 256) ? 1u : 0u;
}

cudaError_t launch_compress_ws(const void *in, uint64_t n, int dtype, uint64_t e_bits, uint32_t block,
                               void *out, void *ws, uint64_t *d_result, cudaStream_t stream, Clear clear) {
    CField one;
    fill_compress_field(&one, in, n, dtype, e_bits, block, out, ws, d_result, 0);
    Workspace *w = reinterpret_cast<Workspace *>(ws);
    CompressLaunch lc;
    lc.fields = nullptr;
    lc.nfields = 1;
    lc.total_tiles = one.g.ntiles;
    lc.ticket = &w->ticket;
    lc.done = &w->done;
    lc.err = &w->err;
    lc.lookback_ns = 1000ull * wait_limit_from_env("SZX_LOOKBACK_US", 1000000u);
    lc.copy_ns = 1000ull * wait_limit_from_env("SZX_COPY_US", 1000000u);
    // the counters and look-back flags start at zero (workspace_bytes is a
    // multiple of 8)
    if (clear == Clear::automatic) clear = one.g.ntiles >= kClearKernelMinTiles ? Clear::kernel : Clear::memset;
    if (clear == Clear::memset) {
        const cudaError_t err = cudaMemsetAsync(ws, 0, workspace_bytes(one.g.ntiles), stream);
        if (err != cudaSuccess) return err;
        return dispatch(dtype, block, 8, one, lc, 0, false, stream);
    }
    // the kernel starts behind the clear
    cudaError_t err = launch_clear_words(static_cast<uint32_t *>(ws), workspace_bytes(one.g.ntiles) / 4, stream);
    if (err != cudaSuccess) return err;
    return dispatch(dtype, block, 8, one, lc, 0, true, stream);
}

cudaError_t launch_compress_batch(const void *d_fields, uint32_t nfields, uint64_t total_tiles, uint32_t *d_counters,
                                  int dtype, uint32_t block, int ctas_per_sm, int nw, bool pdl, cudaStream_t stream) {
    CField one;
    std::memset(&one, 0, sizeof(one));
    CompressLaunch lc;
    lc.fields = static_cast<const CField *>(d_fields);
    lc.nfields = nfields;
    lc.total_tiles = total_tiles;
    lc.ticket = d_counters;
    lc.done = d_counters + 1;
    lc.err = d_counters + 2;
    lc.lookback_ns = 1000ull * wait_limit_from_env("SZX_LOOKBACK_US", 1000000u);
    lc.copy_ns = 1000ull * wait_limit_from_env("SZX_COPY_US", 1000000u);
    return dispatch(dtype, block, nw, one, lc, ctas_per_sm, pdl, stream);
}

// ---------------------------------------------------------------------------

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}
}  // namespace

bool encode_row_map(CUtensorMap *tm, const void *base, uint64_t rows, uint32_t box_rows) {
    std::memset(tm, 0, sizeof(*tm));
    if (rows == 0 || rows >= (1ull << 31)) return false;
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {32, rows};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {32, box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace szx
