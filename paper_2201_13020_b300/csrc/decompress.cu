// decompress.cu -- SZx decompression kernel for sm_103a.
//
// One CTA decodes one tile.  The tile index written by the compressor gives
// the record's offset directly, so tiles decode independently: no device-wide
// scan is left for decompression (the paper's GPU decoder, Sec. V-B, needs a
// prefix scan of the mid-byte counts first).  Per tile:
//   1. one thread bulk-copies the record into shared memory (TMA,
//      cp.async.bulk + mbarrier); the state bits and mu values of the tile are
//      loaded alongside;
//   2. warp 0 ranks the non-constant blocks; each warp reads the reqBits byte
//      and lead codes of its blocks and counts their mid bytes; warp 0 scans
//      the counts into mid-byte offsets and checks them against the record
//      size (every read below is inside the record);
//   3. each warp rebuilds its blocks: the own bytes of every value come from
//      the mid-byte planes; a leading byte (one identical to the previous
//      value's) is resolved per byte plane as a segmented "last writer" scan
//      across the warp -- a ballot of the lanes that own a byte of that plane
//      and a shuffle from the nearest such lane below -- which is the paper's
//      index propagation (Sec. V-B) done in one step per plane; then
//      v' = t << s and d' = RN(v' + mu).
#include "szx_device.cuh"
#include "szx_launch.h"

#include <type_traits>

namespace szx {

struct DecompressArgs {
    const uint8_t *in;
    uint64_t in_bytes;
    uint8_t *out;
    uint32_t *status;
    Geometry g;
    uint64_t rec_total;
    uint32_t dtype;
    uint32_t check_header;  // re-check the stream header on the device
    uint64_t copy_ns;       // wall-time limit of the record copy wait
    uint64_t total_bytes;
};

__device__ __forceinline__ void flag_status(uint32_t *status, uint32_t code) {
    if (status) atomicMax(status, code);
}

template <typename U, int VPL>
__device__ __forceinline__ void store_out(U *p, const U (&x)[VPL], int nvalid) {
    constexpr int bytes = VPL * (int)sizeof(U);
    if (nvalid == VPL) {
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
    } else {
#pragma unroll
        for (int m = 0; m < VPL; ++m)
            if (m < nvalid) p[m] = x[m];
    }
}

template <int VPL>
using DCodeT = std::conditional_t<(VPL > 16), uint64_t, uint32_t>;

template <int VPL>
__device__ __forceinline__ DCodeT<VPL> lane_codes(const uint8_t *slot) {
    const int lane = lane_id();
    if constexpr (VPL >= 4) {
        constexpr int nb = VPL / 4;
        DCodeT<VPL> c = 0;
#pragma unroll
        for (int i = 0; i < nb; ++i) c |= (DCodeT<VPL>)slot[lane * nb + i] << (8 * i);
        return c;
    } else if constexpr (VPL == 2) {
        return (slot[lane >> 1] >> (4 * (lane & 1))) & 0xFu;
    } else {
        return (slot[lane >> 2] >> (2 * (lane & 3))) & 0x3u;
    }
}

template <int VPL>
struct DPlanePack {
    using T = std::conditional_t<(VPL > 16), uint64_t, uint32_t>;
    static constexpr int PB = VPL > 16 ? 16 : 10;
    static constexpr T one3 = (T(1) << (2 * PB)) | (T(1) << PB) | T(1);
    __device__ __forceinline__ static T inc(int L) { return (one3 >> (PB * L)) << (PB * L); }
    __device__ __forceinline__ static uint32_t field(T v, int j) {
        return (uint32_t)(v >> (PB * j)) & ((1u << PB) - 1);
    }
};

template <typename T, int VPL>
__global__ void __launch_bounds__(kThreads) decompress_kernel(DecompressArgs a) {
    using F = Fmt<T>;
    using U = typename F::U;
    constexpr int w = F::w;
    constexpr int W = F::W;

    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_size, s_bad, s_nn, s_mid;

    const Geometry &g = a.g;
    const uint32_t b = g.b, G = g.G;
    const DecompressSmem L = decompress_smem(G, b, w);
    uint8_t *sm_rec = smem + L.rec;
    U *sm_mu = reinterpret_cast<U *>(smem + L.mu);
    uint8_t *sm_state = smem + L.state;
    uint8_t *sm_req = smem + L.req;
    uint32_t *sm_mk = reinterpret_cast<uint32_t *>(smem + L.mk);
    uint32_t *sm_rank = reinterpret_cast<uint32_t *>(smem + L.rank);
    uint32_t *sm_midoff = reinterpret_cast<uint32_t *>(smem + L.midoff);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tile = blockIdx.x;
    const uint64_t k0 = (uint64_t)tile * G;
    const uint32_t Gt = (uint32_t)min_u64(G, g.nb - k0);
    const uint32_t rec_max = record_max_bytes(G, b, w);

    // ---- 1. record, state bits and mu of the tile -------------------------
    if (tid == 0) {
        uint32_t bad = 0;
        if (a.check_header && tile == 0) {
            const uint32_t *h32 = reinterpret_cast<const uint32_t *>(a.in);
            const uint64_t *h64 = reinterpret_cast<const uint64_t *>(a.in);
            if (h32[0] != kMagic || (h32[1] & 0xFFFFu) != (kVersion | (a.dtype << 8)) || h32[2] != b ||
                h32[3] != G || h64[2] != g.n || h64[7] != a.total_bytes)
                bad = 1;
        }
        const uint64_t *idx = reinterpret_cast<const uint64_t *>(a.in + g.off_index);
        const uint64_t r0 = idx[tile], r1 = idx[tile + 1];
        if (r0 > r1 || r1 > a.rec_total || (r0 & 15) || (r1 & 15) || r1 - r0 > rec_max) bad = 1;
        if (tile == g.ntiles - 1 && r1 != a.rec_total) bad = 1;
        const uint32_t size = bad ? 0u : (uint32_t)(r1 - r0);
        s_size = size;
        s_bad = bad;
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (size) {
            mbar_arrive_expect_tx(&bar, size);
            bulk_g2s(sm_rec, a.in + g.off_rec + r0, size, &bar);
        }
    }
    {
        const uint8_t *st = a.in + g.off_state + k0 / 8;
        for (uint32_t i = tid; i < (Gt + 7) / 8; i += kThreads) sm_state[i] = st[i];
        const U *mu = reinterpret_cast<const U *>(a.in + g.off_mu) + k0;
        for (uint32_t i = tid; i < Gt; i += kThreads) sm_mu[i] = mu[i];
    }
    __syncthreads();
    const uint32_t size = s_size;
    if (size && !mbar_wait_bounded(&bar, 0, a.copy_ns)) s_bad = 2;
    __syncthreads();

    // ---- 2. ranks, mid-byte counts, offsets -------------------------------
    if (warp == 0) {
        const uint32_t per = (Gt + 31) / 32;
        const uint32_t lo = min(lane * per, Gt), hi = min(lo + per, Gt);
        uint32_t c = 0;
        for (uint32_t kk = lo; kk < hi; ++kk) c += (sm_state[kk >> 3] >> (kk & 7)) & 1u;
        uint32_t tot;
        uint32_t e = warp_exclusive_scan(c, &tot);
        for (uint32_t kk = lo; kk < hi; ++kk) {
            sm_rank[kk] = e;
            e += (sm_state[kk >> 3] >> (kk & 7)) & 1u;
        }
        if (lane == 0) {
            s_nn = tot;
            if ((uint64_t)tot * (b / 4 + 1) > size) s_bad |= 1;
        }
    }
    __syncthreads();
    const uint32_t nn_t = s_nn;
    if (!s_bad) {
        for (uint32_t kk = warp; kk < Gt; kk += kWarps) {
            if (!((sm_state[kk >> 3] >> (kk & 7)) & 1u)) {
                if (lane == 0) sm_mk[kk] = 0;
                continue;
            }
            const uint32_t rank = sm_rank[kk];
            const int len = (int)min_u64(b, g.n - (k0 + kk) * b);
            const int rq = sm_rec[nn_t * (b / 4) + rank];
            uint32_t mk;
            bool ok = true;
            if (rq == 0xFF) {
                mk = (uint32_t)len * w;
            } else {
                ok = rq >= 1 + F::E && rq <= W;
                const int s = (8 - (rq & 7)) & 7;
                const int q = (rq + s) >> 3;
                const int lmax = q < 3 ? q : 3;
                const DCodeT<VPL> codes = lane_codes<VPL>(sm_rec + rank * (b / 4));
                uint32_t cnt = 0;
#pragma unroll
                for (int m = 0; m < VPL; ++m) {
                    const int l = (int)(codes >> (2 * m)) & 3;
                    const bool valid = lane * VPL + m < len;
                    if (valid) {
                        ok = ok && l <= lmax;
                        cnt += (uint32_t)(q - l);
                    } else {
                        ok = ok && l == 0;
                    }
                }
                ok = __all_sync(kFull, ok);
                mk = __reduce_add_sync(kFull, ok ? cnt : 0u);
            }
            if (lane == 0) {
                sm_req[kk] = (uint8_t)rq;
                sm_mk[kk] = mk;
                if (!ok) s_bad |= 1;
            }
        }
    }
    __syncthreads();
    if (warp == 0 && !s_bad) {
        const uint32_t per = (Gt + 31) / 32;
        const uint32_t lo = min(lane * per, Gt), hi = min(lo + per, Gt);
        uint32_t c = 0;
        for (uint32_t kk = lo; kk < hi; ++kk) c += sm_mk[kk];
        uint32_t tot;
        uint32_t e = warp_exclusive_scan(c, &tot);
        for (uint32_t kk = lo; kk < hi; ++kk) {
            sm_midoff[kk] = e;
            e += sm_mk[kk];
        }
        if (lane == 0) {
            s_mid = tot;
            const uint64_t used = (uint64_t)nn_t * (b / 4 + 1) + tot;
            if (pad16(used) != size) s_bad |= 1;
        }
    }
    __syncthreads();
    if (!s_bad) {
        // the record's pad bytes must be zero
        const uint32_t used = nn_t * (b / 4 + 1) + s_mid;
        for (uint32_t i = used + tid; i < size; i += kThreads)
            if (sm_rec[i]) s_bad |= 1;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) flag_status(a.status, s_bad & 2 ? 6u : 3u);
        if (tid == 0 && size && (s_bad & 2)) mbar_wait_bounded(&bar, 0, a.copy_ns);
        return;
    }

    // ---- 3. decode ---------------------------------------------------------
    const uint32_t mid_base = nn_t * (b / 4 + 1);
    U *out = reinterpret_cast<U *>(a.out);
    for (uint32_t kk = warp; kk < Gt; kk += kWarps) {
        const uint64_t first = (k0 + kk) * b;
        const int len = (int)min_u64(b, g.n - first);
        const int nvalid = max(0, min(VPL, len - lane * VPL));
        U *dst = out + first + lane * VPL;
        U x[VPL];
        const U mu_bits = sm_mu[kk];
        if (!((sm_state[kk >> 3] >> (kk & 7)) & 1u)) {
#pragma unroll
            for (int m = 0; m < VPL; ++m) x[m] = mu_bits;
            store_out<U, VPL>(dst, x, nvalid);
            continue;
        }
        const uint32_t rank = sm_rank[kk];
        const uint8_t *mid = sm_rec + mid_base + sm_midoff[kk];
        const int rq = sm_req[kk];
        if (rq == 0xFF) {
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                U u = 0;
                if (m < nvalid) {
                    const uint8_t *p = mid + (size_t)(lane * VPL + m) * w;
#pragma unroll
                    for (int i = 0; i < w; ++i) u |= (U)p[i] << (8 * i);
                }
                x[m] = u;
            }
            store_out<U, VPL>(dst, x, nvalid);
            continue;
        }
        const int s = (8 - (rq & 7)) & 7;
        const int q = (rq + s) >> 3;
        const int lmax = q < 3 ? q : 3;
        const DCodeT<VPL> codes = lane_codes<VPL>(sm_rec + rank * (b / 4));
        int Lm[VPL];
        bool valid[VPL];
        typename DPlanePack<VPL>::T cnt = 0;
#pragma unroll
        for (int m = 0; m < VPL; ++m) {
            valid[m] = m < nvalid;
            Lm[m] = (int)(codes >> (2 * m)) & 3;
            if (valid[m]) cnt += DPlanePack<VPL>::inc(Lm[m]);
        }
        typename DPlanePack<VPL>::T tot;
        const typename DPlanePack<VPL>::T off = warp_exclusive_scan(cnt, &tot);
        const uint32_t n0 = DPlanePack<VPL>::field(tot, 0), n1 = DPlanePack<VPL>::field(tot, 1),
                       n2 = DPlanePack<VPL>::field(tot, 2);
        const uint32_t P[3] = {0u, n0, n0 + n1};
        // own bytes from the planes
        U own[VPL];
#pragma unroll
        for (int m = 0; m < VPL; ++m) own[m] = 0;
        const int sparse = q < 3 ? q : 3;
        for (int j = 0; j < sparse; ++j) {
            uint32_t pos = P[j] + DPlanePack<VPL>::field(off, j);
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                if (valid[m] && Lm[m] <= j) own[m] |= (U)mid[pos++] << (W - 8 - 8 * j);
            }
        }
        for (int j = 3; j < q; ++j) {
            const uint8_t *plane = mid + n0 + n1 + n2 + (uint32_t)(j - 3) * len + lane * VPL;
#pragma unroll
            for (int m = 0; m < VPL; ++m)
                if (valid[m]) own[m] |= (U)plane[m] << (W - 8 - 8 * j);
        }
        // leading bytes: per plane j < lmax, the nearest earlier owner
        U incoming = 0;
        for (int j = 0; j < lmax; ++j) {
            bool has = false;
            uint32_t last = 0;
#pragma unroll
            for (int m = 0; m < VPL; ++m) {
                if (valid[m] && Lm[m] <= j) {
                    has = true;
                    last = (uint32_t)(own[m] >> (W - 8 - 8 * j)) & 0xFFu;
                }
            }
            const uint32_t below = __ballot_sync(kFull, has) & ((1u << lane) - 1u);
            const int src = below ? 31 - __clz(below) : 0;
            uint32_t byte = __shfl_sync(kFull, last, src);
            if (!below) byte = 0;
            incoming |= (U)byte << (W - 8 - 8 * j);
        }
        U prev = incoming;
        const T mu = F::from(mu_bits);
#pragma unroll
        for (int m = 0; m < VPL; ++m) {
            const int l = Lm[m];
            const U hi = l ? ~(U)0 << (W - 8 * l) : (U)0;
            const U t = own[m] | (prev & hi);
            prev = t;
            x[m] = F::bits(F::add(F::from((U)(t << s)), mu));
        }
        store_out<U, VPL>(dst, x, nvalid);
    }
}

// ---------------------------------------------------------------------------

template <typename T, int VPL>
static cudaError_t launch_t(const DecompressArgs &a, cudaStream_t stream) {
    const DecompressSmem L = decompress_smem(a.g.G, a.g.b, Fmt<T>::w);
    auto kern = decompress_kernel<T, VPL>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)a.g.ntiles, kThreads, L.total, stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_vpl(const DecompressArgs &a, cudaStream_t stream) {
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

cudaError_t launch_decompress(const void *in, uint64_t in_bytes, uint64_t total_bytes, uint64_t n, int dtype,
                              uint32_t block, void *out, uint32_t *d_status, bool check_header,
                              cudaStream_t stream) {
    DecompressArgs a;
    a.in = static_cast<const uint8_t *>(in);
    a.in_bytes = in_bytes;
    a.out = static_cast<uint8_t *>(out);
    a.status = d_status;
    a.g = make_geometry(n, block, dtype == 0 ? 4 : 8);
    a.rec_total = total_bytes - a.g.off_rec;
    a.dtype = (uint32_t)dtype;
    a.check_header = check_header ? 1u : 0u;
    a.total_bytes = total_bytes;
    a.copy_ns = 1000ull * wait_limit_from_env("SZX_COPY_US", 1000000u);
    return dtype == 0 ? launch_vpl<float>(a, stream) : launch_vpl<double>(a, stream);
}

}  // namespace szx
