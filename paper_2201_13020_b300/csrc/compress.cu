// compress.cu -- single-pass SZx compression kernel for sm_103a.
//
// One CTA compresses one tile of G consecutive blocks (32 KiB of input) and
// emits the tile's record; tiles are taken in ticket order so that the
// decoupled look-back over tile record sizes (the device-wide exclusive scan
// that places each record, cf. the prefix scan of Sec. V-B) always waits on
// tiles that are already running.  Per tile:
//   1. one thread bulk-copies the tile's input into shared memory (TMA,
//      cp.async.bulk + mbarrier);
//   2. each warp encodes whole blocks (Algorithm 1): min/max of the block as
//      order-preserving integer keys with warp reductions, mu and r, the exact
//      constant test, reqBits (Eq. 3), the Eq. 4 shift and truncation with the
//      exact per-value bound check, the XOR identical-leading-byte codes, and
//      the block's mid-byte count; the truncated words overwrite the input in
//      shared memory;
//   3. warp 0 scans the blocks of the tile (non-constant rank, mid-byte
//      offsets) and the tile publishes its record size;
//   4. all warps write the record into shared memory: lead codes, reqBits
//      bytes, and the mid-byte planes (plane j = byte j of each value whose
//      identical-leading-byte count is <= j, ascending value index);
//   5. one thread finishes the look-back, writes the tile index entry, and
//      bulk-stores the record to its offset.
#include "szx_device.cuh"
#include "szx_launch.h"

#include <limits>
#include <type_traits>

namespace szx {

struct CompressArgs {
    const uint8_t *in;
    uint8_t *out;
    Workspace *ws;
    uint64_t *lookback;
    uint64_t *d_result;
    Geometry g;
    uint64_t e_bits;
    uint32_t dtype;
    uint32_t spin_limit;
};

template <typename U, int VPL>
__device__ __forceinline__ void load_lane(const U *p, U (&x)[VPL]) {
    constexpr int bytes = VPL * (int)sizeof(U);
    if constexpr (bytes % 16 == 0) {
#pragma unroll
        for (int i = 0; i < bytes / 16; ++i) {
            uint4 v = reinterpret_cast<const uint4 *>(p)[i];
            const U *u = reinterpret_cast<const U *>(&v);
#pragma unroll
            for (int j = 0; j < 16 / (int)sizeof(U); ++j) x[i * (16 / sizeof(U)) + j] = u[j];
        }
    } else if constexpr (bytes == 8) {
        uint2 v = *reinterpret_cast<const uint2 *>(p);
        const U *u = reinterpret_cast<const U *>(&v);
#pragma unroll
        for (int j = 0; j < VPL; ++j) x[j] = u[j];
    } else {
        x[0] = p[0];
    }
}

template <typename U, int VPL>
__device__ __forceinline__ void store_lane(U *p, const U (&x)[VPL]) {
    constexpr int bytes = VPL * (int)sizeof(U);
    if constexpr (bytes % 16 == 0) {
#pragma unroll
        for (int i = 0; i < bytes / 16; ++i) {
            uint4 v;
            U *u = reinterpret_cast<U *>(&v);
#pragma unroll
            for (int j = 0; j < 16 / (int)sizeof(U); ++j) u[j] = x[i * (16 / sizeof(U)) + j];
            reinterpret_cast<uint4 *>(p)[i] = v;
        }
    } else if constexpr (bytes == 8) {
        uint2 v;
        U *u = reinterpret_cast<U *>(&v);
#pragma unroll
        for (int j = 0; j < VPL; ++j) u[j] = x[j];
        *reinterpret_cast<uint2 *>(p) = v;
    } else {
        p[0] = x[0];
    }
}

// Lead codes of one lane (2 bits per value, value m at bits 2m) to and from
// the block's b/4-byte code slot (value i at byte i/4, bits 2(i%4)).
template <int VPL>
using CodeT = std::conditional_t<(VPL > 16), uint64_t, uint32_t>;

template <int VPL>
__device__ __forceinline__ void put_codes(uint8_t *slot, CodeT<VPL> c) {
    const int lane = lane_id();
    if constexpr (VPL >= 4) {
        constexpr int nb = VPL / 4;
        if constexpr (nb == 1) slot[lane] = (uint8_t)c;
        else if constexpr (nb == 2) reinterpret_cast<uint16_t *>(slot)[lane] = (uint16_t)c;
        else if constexpr (nb == 4) reinterpret_cast<uint32_t *>(slot)[lane] = (uint32_t)c;
        else reinterpret_cast<uint64_t *>(slot)[lane] = (uint64_t)c;
    } else if constexpr (VPL == 2) {
        uint32_t hi = __shfl_down_sync(kFull, (uint32_t)c, 1);
        if ((lane & 1) == 0) slot[lane >> 1] = (uint8_t)(c | (hi << 4));
    } else {
        uint32_t c1 = __shfl_down_sync(kFull, (uint32_t)c, 1);
        uint32_t c2 = __shfl_down_sync(kFull, (uint32_t)c, 2);
        uint32_t c3 = __shfl_down_sync(kFull, (uint32_t)c, 3);
        if ((lane & 3) == 0) slot[lane >> 2] = (uint8_t)(c | (c1 << 2) | (c2 << 4) | (c3 << 6));
    }
}

template <int VPL>
__device__ __forceinline__ CodeT<VPL> get_codes(const uint8_t *slot) {
    const int lane = lane_id();
    if constexpr (VPL >= 4) {
        constexpr int nb = VPL / 4;
        if constexpr (nb == 1) return slot[lane];
        else if constexpr (nb == 2) return reinterpret_cast<const uint16_t *>(slot)[lane];
        else if constexpr (nb == 4) return reinterpret_cast<const uint32_t *>(slot)[lane];
        else return reinterpret_cast<const uint64_t *>(slot)[lane];
    } else if constexpr (VPL == 2) {
        return (slot[lane >> 1] >> (4 * (lane & 1))) & 0xFu;
    } else {
        return (slot[lane >> 2] >> (2 * (lane & 3))) & 0x3u;
    }
}

// Per-lane counts of values with L <= j for the three sparse planes j = 0,1,2,
// packed in fields of PB bits (a plane of a block holds at most b <= 1024).
template <int VPL>
struct PlanePack {
    using T = std::conditional_t<(VPL > 16), uint64_t, uint32_t>;
    static constexpr int PB = VPL > 16 ? 16 : 10;
    static constexpr T one3 = (T(1) << (2 * PB)) | (T(1) << PB) | T(1);
    __device__ __forceinline__ static T inc(int L) { return (one3 >> (PB * L)) << (PB * L); }
    __device__ __forceinline__ static uint32_t field(T v, int j) {
        return (uint32_t)(v >> (PB * j)) & ((1u << PB) - 1);
    }
};

template <typename U>
__device__ __forceinline__ uint32_t byte_of(U t, int j) {
    constexpr int W = 8 * sizeof(U);
    return (uint32_t)(t >> (W - 8 - 8 * j)) & 0xFFu;
}

template <typename T, int VPL>
__global__ void __launch_bounds__(kThreads) compress_kernel(CompressArgs a) {
    using F = Fmt<T>;
    using U = typename F::U;
    using S = typename F::S;
    constexpr int w = F::w;
    constexpr int W = F::W;

    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tile, s_nn, s_mid, s_nraw, s_nesc, s_rec, s_fail;
    __shared__ uint64_t s_excl;

    const Geometry &g = a.g;
    const uint32_t b = g.b, G = g.G;
    const CompressSmem L = compress_smem(G, b, w);
    uint8_t *sm_in = smem + L.in;
    uint8_t *sm_rec = smem + L.rec;
    uint8_t *sm_lead = smem + L.lead;
    U *sm_mu = reinterpret_cast<U *>(smem + L.mu);
    uint8_t *sm_kind = smem + L.kind;
    uint8_t *sm_req = smem + L.req;
    uint32_t *sm_mk = reinterpret_cast<uint32_t *>(smem + L.mk);
    uint32_t *sm_rank = reinterpret_cast<uint32_t *>(smem + L.rank);
    uint32_t *sm_midoff = reinterpret_cast<uint32_t *>(smem + L.midoff);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- 1. ticket and bulk load of the tile's input ----------------------
    if (tid == 0) {
        s_tile = atomicAdd(&a.ws->ticket, 1u);
        s_fail = 0;
        s_nesc = 0;
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t k0 = (uint64_t)tile * G;
    const uint32_t Gt = (uint32_t)min_u64(G, g.nb - k0);
    const uint64_t v0 = k0 * b;
    const uint32_t tile_vals = (uint32_t)min_u64((uint64_t)G * b, g.n - v0);
    const uint32_t tile_bytes = tile_vals * w;
    const uint32_t bulk_bytes = tile_bytes & ~15u;
    if (tid == 0 && bulk_bytes) {
        mbar_arrive_expect_tx(&bar, bulk_bytes);
        bulk_g2s(sm_in, a.in + v0 * w, bulk_bytes, &bar);
    }
    // ragged tail (last tile only): plain loads, then zero the unused words
    for (uint32_t i = bulk_bytes + tid; i < tile_bytes; i += kThreads) sm_in[i] = a.in[v0 * w + i];
    for (uint32_t i = tile_bytes + tid; i < G * b * w; i += kThreads) sm_in[i] = 0;
    if (bulk_bytes && !mbar_wait_bounded(&bar, 0, 1u << 24)) s_fail = 1;
    __syncthreads();
    // (a bulk copy that never completed leaves s_fail set: the tile then
    // publishes an empty record and the call reports SZX_ERR_TIMEOUT)

    const T e = F::from((U)a.e_bits);

    // ---- 2. per-warp block encoding ---------------------------------------
    for (uint32_t kk = warp; kk < Gt && !s_fail; kk += kWarps) {
        const uint64_t first = (k0 + kk) * b;
        const int len = (int)min_u64(b, g.n - first);
        U *vp = reinterpret_cast<U *>(sm_in) + (size_t)kk * b + lane * VPL;
        U x[VPL];
        load_lane<U, VPL>(vp, x);
        bool valid[VPL];
#pragma unroll
        for (int m = 0; m < VPL; ++m) valid[m] = lane * VPL + m < len;

        // block statistics: min / max as order-preserving keys
        S kmin = std::numeric_limits<S>::max(), kmax = std::numeric_limits<S>::min();
#pragma unroll
        for (int m = 0; m < VPL; ++m) {
            if (valid[m]) {
                S kx = F::key(x[m]);
                kmin = kx < kmin ? kx : kmin;
                kmax = kx > kmax ? kx : kmax;
            }
        }
        kmin = warp_min(kmin);
        kmax = warp_max(kmax);
        const bool all_finite = kmin > F::kKeyNegInf && kmax < F::kKeyPosInf;
        const T mn = F::from(F::unkey(kmin)), mx = F::from(F::unkey(kmax));
        const T r = F::half(F::sub(mx, mn));
        const T mu = F::add(mn, r);

        int kind = kRaw, req = 0xFF, escalated = 0;
        uint32_t mk = (uint32_t)len * w;
        if (all_finite && F::finite(F::bits(r)) && F::finite(F::bits(mu))) {
            if (within(mx, mu, e) && within(mn, mu, e)) {
                kind = kConst;
                mk = 0;
            } else {
                // Eq. 3 with sign and exponent always kept
                int R = F::expo(F::bits(r)) - F::expo(F::bits(e));
                R = R < 0 ? 0 : (R > F::M ? F::M : R);
                const int req0 = 1 + F::E + R;
                U v[VPL];
#pragma unroll
                for (int m = 0; m < VPL; ++m) v[m] = F::bits(F::sub(F::from(x[m]), mu));
                int rq = req0;
                for (; rq <= W; ++rq) {
                    const int s = (8 - (rq & 7)) & 7;
                    const U mask = top_bytes_mask<U>((rq + s) >> 3);
                    bool ok = true;
#pragma unroll
                    for (int m = 0; m < VPL; ++m) {
                        if (valid[m]) {
                            const U t = (v[m] >> s) & mask;
                            const T dp = F::add(F::from((U)(t << s)), mu);
                            ok = ok && within(F::from(x[m]), dp, e);
                        }
                    }
                    if (__all_sync(kFull, ok)) break;
                }
                if (rq <= W) {
                    kind = kNonConst;
                    req = rq;
                    escalated = rq > req0;
                    const int s = (8 - (rq & 7)) & 7;
                    const int q = (rq + s) >> 3;
                    const U mask = top_bytes_mask<U>(q);
                    const int lmax = q < 3 ? q : 3;
                    U t[VPL];
#pragma unroll
                    for (int m = 0; m < VPL; ++m) t[m] = valid[m] ? (v[m] >> s) & mask : U(0);
                    U prev = __shfl_up_sync(kFull, t[VPL - 1], 1);
                    if (lane == 0) prev = 0;
                    CodeT<VPL> codes = 0;
                    uint32_t cnt = 0;
#pragma unroll
                    for (int m = 0; m < VPL; ++m) {
                        int l = F::clz(t[m] ^ prev) >> 3;
                        l = l < lmax ? l : lmax;
                        if (!valid[m]) l = 0;
                        codes |= (CodeT<VPL>)l << (2 * m);
                        cnt += valid[m] ? (uint32_t)(q - l) : 0u;
                        prev = t[m];
                    }
                    put_codes<VPL>(sm_lead + (size_t)kk * (b / 4), codes);
                    store_lane<U, VPL>(vp, t);
                    mk = __reduce_add_sync(kFull, cnt);
                }
            }
        }
        if (lane == 0) {
            sm_kind[kk] = (uint8_t)kind;
            sm_req[kk] = (uint8_t)req;
            sm_mk[kk] = mk;
            sm_mu[kk] = (kind == kRaw) ? U(0) : F::bits(mu);
            if (escalated) atomicAdd(&s_nesc, 1u);
        }
    }
    __syncthreads();

    // ---- 3. tile scan: non-constant ranks and mid-byte offsets -------------
    if (warp == 0) {
        const uint32_t per = (Gt + 31) / 32;
        const uint32_t lo = min(lane * per, Gt), hi = min(lo + per, Gt);
        uint32_t c_nn = 0, c_mid = 0, c_raw = 0;
        for (uint32_t kk = lo; kk < hi; ++kk) {
            if (sm_kind[kk] != kConst) {
                c_nn += 1;
                c_mid += sm_mk[kk];
                c_raw += sm_kind[kk] == kRaw;
            }
        }
        uint32_t t_nn, t_mid, t_raw;
        uint32_t e_nn = warp_exclusive_scan(c_nn, &t_nn);
        uint32_t e_mid = warp_exclusive_scan(c_mid, &t_mid);
        warp_exclusive_scan(c_raw, &t_raw);
        for (uint32_t kk = lo; kk < hi; ++kk) {
            sm_rank[kk] = e_nn;
            sm_midoff[kk] = e_mid;
            if (sm_kind[kk] != kConst) {
                e_nn += 1;
                e_mid += sm_mk[kk];
            }
        }
        if (lane == 0) {
            s_nn = t_nn;
            s_mid = t_mid;
            s_nraw = t_raw;
            const uint32_t used = t_nn * (b / 4 + 1) + t_mid;
            s_rec = s_fail ? 0u : (uint32_t)pad16(used);
            // publish this tile's aggregate so later tiles can look back
            st_release_u64(&a.lookback[tile], kFlagAgg | s_rec);
        }
    }
    __syncthreads();

    // ---- 4. the record in shared memory ------------------------------------
    const uint32_t nn_t = s_nn;
    const uint32_t mid_base = nn_t * (b / 4 + 1);
    if (!s_fail) {
        for (uint32_t kk = warp; kk < Gt; kk += kWarps) {
            const int kind = sm_kind[kk];
            if (kind == kConst) continue;
            const uint32_t rank = sm_rank[kk];
            const uint64_t first = (k0 + kk) * b;
            const int len = (int)min_u64(b, g.n - first);
            uint8_t *lead_dst = sm_rec + rank * (b / 4);
            const uint8_t *lead_src = sm_lead + (size_t)kk * (b / 4);
            for (uint32_t i = lane; i < b / 4; i += 32) lead_dst[i] = kind == kRaw ? 0 : lead_src[i];
            if (lane == 0) sm_rec[nn_t * (b / 4) + rank] = sm_req[kk];
            uint8_t *mid = sm_rec + mid_base + sm_midoff[kk];
            if (kind == kRaw) {
                const uint8_t *src = sm_in + (size_t)kk * b * w;
                for (uint32_t i = lane; i < (uint32_t)len * w; i += 32) mid[i] = src[i];
                continue;
            }
            const int rq = sm_req[kk];
            const int s = (8 - (rq & 7)) & 7;
            const int q = (rq + s) >> 3;
            U t[VPL];
            load_lane<U, VPL>(reinterpret_cast<const U *>(sm_in) + (size_t)kk * b + lane * VPL, t);
            const CodeT<VPL> codes = get_codes<VPL>(lead_src);
            int Lm[VPL];
            bool valid[VPL];
            typename PlanePack<VPL>::T cnt = 0;
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                valid[m] = lane * VPL + m < len;
                Lm[m] = (int)(codes >> (2 * m)) & 3;
                if (valid[m]) cnt += PlanePack<VPL>::inc(Lm[m]);
            }
            typename PlanePack<VPL>::T tot;
            const typename PlanePack<VPL>::T off = warp_exclusive_scan(cnt, &tot);
            const uint32_t n0 = PlanePack<VPL>::field(tot, 0), n1 = PlanePack<VPL>::field(tot, 1),
                           n2 = PlanePack<VPL>::field(tot, 2);
            const uint32_t P[3] = {0u, n0, n0 + n1};
            const int sparse = q < 3 ? q : 3;
            for (int j = 0; j < sparse; ++j) {
                uint32_t pos = P[j] + PlanePack<VPL>::field(off, j);
#pragma unroll
                for (int m = 0; m < VPL; ++m) {
                    if (valid[m] && Lm[m] <= j) mid[pos++] = (uint8_t)byte_of(t[m], j);
                }
            }
            // planes j >= 3 hold every value (L <= 3 <= j)
            for (int j = 3; j < q; ++j) {
                uint8_t *plane = mid + n0 + n1 + n2 + (uint32_t)(j - 3) * len + lane * VPL;
#pragma unroll
                for (int m = 0; m < VPL; ++m)
                    if (valid[m]) plane[m] = (uint8_t)byte_of(t[m], j);
            }
        }
        // zero pad of the record
        const uint32_t used = mid_base + s_mid;
        for (uint32_t i = used + tid; i < s_rec; i += kThreads) sm_rec[i] = 0;
    }
    __syncthreads();

    // ---- 5. look-back, index entry, record store ---------------------------
    if (tid == 0) {
        if (s_fail) atomicOr(&a.ws->err, kErrTimeout);
        uint64_t excl = 0;
        uint32_t spins = 0;
        bool timed_out = false;
        for (int64_t j = (int64_t)tile - 1; j >= 0;) {
            const uint64_t wv = ld_acquire_u64(&a.lookback[j]);
            const uint64_t flag = wv & ~kValueMask;
            if (flag == 0) {
                if (++spins > a.spin_limit) {
                    timed_out = true;
                    break;
                }
                __nanosleep(32);
                continue;
            }
            excl += wv & kValueMask;
            if (flag == kFlagPrefix) break;
            --j;
        }
        if (timed_out) atomicOr(&a.ws->err, kErrTimeout);
        st_release_u64(&a.lookback[tile], kFlagPrefix | (excl + s_rec));
        s_excl = excl;
        uint8_t *idx = a.out + g.off_index;
        reinterpret_cast<uint64_t *>(idx)[tile] = excl;
        if (tile == g.ntiles - 1) {
            const uint64_t rec_total = excl + s_rec;
            reinterpret_cast<uint64_t *>(idx)[g.ntiles] = rec_total;
            // zero pads of the fixed sections
            const uint64_t state_end = g.off_state + (g.nb + 7) / 8;
            for (uint64_t i = state_end; i < g.off_mu; ++i) a.out[i] = 0;
            for (uint64_t i = g.off_mu + g.nb * w; i < g.off_index; ++i) a.out[i] = 0;
            for (uint64_t i = g.off_index + 8 * (g.ntiles + 1); i < g.off_rec; ++i) a.out[i] = 0;
        }
    }
    __syncthreads();
    const uint64_t excl = s_excl;
    if (tid == 0 && s_rec) {
        fence_proxy_async_smem();
        bulk_s2g(a.out + g.off_rec + excl, sm_rec, s_rec);
        bulk_commit();
    }
    // state bits and mu values of the tile (fixed positions)
    {
        uint8_t *state = a.out + g.off_state + (size_t)k0 / 8;
        for (uint32_t i = tid; i < (Gt + 7) / 8; i += kThreads) {
            uint32_t byte = 0;
            for (int j = 0; j < 8; ++j) {
                const uint32_t kk = i * 8 + j;
                if (kk < Gt && sm_kind[kk] != kConst) byte |= 1u << j;
            }
            state[i] = (uint8_t)byte;
        }
        U *mu_dst = reinterpret_cast<U *>(a.out + g.off_mu) + k0;
        for (uint32_t i = tid; i < Gt; i += kThreads) mu_dst[i] = sm_mu[i];
    }
    // counters and completion
    if (tid == 0) {
        atomicAdd(&a.ws->nn, (unsigned long long)s_nn);
        atomicAdd(&a.ws->nraw, (unsigned long long)s_nraw);
        atomicAdd(&a.ws->nesc, (unsigned long long)s_nesc);
        __threadfence();
        const uint32_t done = atomicAdd(&a.ws->done, 1u);
        if (done == g.ntiles - 1) {
            // last tile to finish: write the header and the result words
            __threadfence();
            volatile Workspace *ws = a.ws;
            const uint64_t rec_total = reinterpret_cast<volatile uint64_t *>(a.out + g.off_index)[g.ntiles];
            const uint64_t total = g.off_rec + rec_total;
            uint8_t *h = a.out;
            uint32_t *h32 = reinterpret_cast<uint32_t *>(h);
            uint64_t *h64 = reinterpret_cast<uint64_t *>(h);
            h32[0] = kMagic;
            h32[1] = kVersion | (a.dtype << 8);
            h32[2] = b;
            h32[3] = G;
            h64[2] = g.n;
            h64[3] = a.e_bits;
            h64[4] = ws->nn;
            h64[5] = ws->nraw;
            h64[6] = ws->nesc;
            h64[7] = total;
            const uint64_t status = (ws->err & kErrTimeout) ? 6ull : 0ull;
            ws->result[0] = total;
            ws->result[1] = status;
            if (a.d_result) {
                a.d_result[0] = total;
                a.d_result[1] = status;
            }
        }
    }
    // the bulk store must have read the record before the CTA's shared memory
    // is released; a bulk load that timed out gets one more bounded wait
    if (tid == 0) {
        if (s_rec) bulk_wait_read_all();
        if (s_fail) mbar_wait_bounded(&bar, 0, 1u << 24);
    }
}

// ---------------------------------------------------------------------------

template <typename T, int VPL>
static cudaError_t launch_t(const CompressArgs &a, cudaStream_t stream) {
    const CompressSmem L = compress_smem(a.g.G, a.g.b, Fmt<T>::w);
    auto kern = compress_kernel<T, VPL>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)a.g.ntiles, kThreads, L.total, stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_vpl(const CompressArgs &a, cudaStream_t stream) {
    switch (a.g.b) {
        case 32: return launch_t<T, 1>(a, stream);
        case 64: return launch_t<T, 2>(a, stream);
        case 128: return launch_t<T, 4>(a, stream);
        case 256: return launch_t<T, 8>(a, stream);
        case 512: return launch_t<T, 16>(a, stream);
        case 1024: return launch_t<T, 32>(a, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_compress(const void *in, uint64_t n, int dtype, uint64_t e_bits, uint32_t block,
                            void *out, uint64_t ws_offset, uint64_t *d_result, cudaStream_t stream) {
    CompressArgs a;
    a.in = static_cast<const uint8_t *>(in);
    a.out = static_cast<uint8_t *>(out);
    a.g = make_geometry(n, block, dtype == 0 ? 4 : 8);
    a.ws = reinterpret_cast<Workspace *>(a.out + ws_offset);
    a.lookback = reinterpret_cast<uint64_t *>(a.out + ws_offset + kWsHeader);
    a.d_result = d_result;
    a.e_bits = e_bits;
    a.dtype = (uint32_t)dtype;
    a.spin_limit = 1u << 22;
    cudaError_t err = cudaMemsetAsync(a.ws, 0, workspace_bytes(a.g.ntiles), stream);
    if (err != cudaSuccess) return err;
    return dtype == 0 ? launch_vpl<float>(a, stream) : launch_vpl<double>(a, stream);
}

}  // namespace szx
