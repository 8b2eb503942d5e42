// decompress.cu -- SZx decompression kernel for sm_103a.
//
// Persistent CTAs decode tiles of G blocks.  The tile index written by the
// compressor gives each record's offset, so tiles decode independently: no
// device-wide scan is left for decompression (the paper's GPU decoder, Sec.
// V-B, runs a prefix scan of the mid-byte counts first).  Per CTA, three warp
// roles share a ring of three stage buffers through mbarriers:
//   producer (one thread): per tile, bulk-copies (cp.async.bulk) the record,
//     the tile's mu values and a 16-byte-aligned window of its state bits into
//     a stage; the tile index entries are loaded one tile ahead, so no global
//     latency sits between two copies;
//   eight decoding warps: decode the stage's record into registers, then
//     write the values back into the same stage buffer as the output tile, in
//     the 128-byte-swizzled row layout of the TMA tensor store;
//   storer (one thread): stores the tile with a 2-D TMA tensor store (rows of
//     128 bytes), then frees the stage for the producer.
// The decoders therefore touch global memory only for the ragged last row.
//
// Work layout as in the compressor: every lane owns 128 contiguous output
// bytes (32 f32 or 16 f64 values); a block of b values spans LPB = b / VPL
// adjacent lanes.  Per tile:
//   1. every lane ranks its block among the tile's non-constant blocks (a
//      popcount of the tile's state bits), reads its reqBits byte and lead
//      codes, checks them, and counts its mid bytes;
//   2. after one barrier every warp scans the blocks' counts into mid-byte
//      offsets and checks the total against the record size, so that every
//      later read is inside the record;
//   3. every lane rebuilds its values: for each group of four values and each
//      byte plane, the lane's run of own bytes is read with two aligned word
//      loads and a funnel shift and spread to the owning values with a
//      table-driven byte permute.  A leading byte (identical to the previous
//      value's) is resolved per plane: inside a lane a byte permute copies the
//      nearest earlier owner forward, and the carry into a lane is the last
//      own byte of the nearest lower lane of the block that owns one (a ballot
//      and a shuffle) -- the paper's index propagation (Sec. V-B) in one step
//      per plane.  A byte transpose turns planes back into words; then
//      v' = t << s and d' = RN(v' + mu);
//   4. after a second barrier (the record is no longer read) the values go to
//      the stage buffer and the storer takes over.
#include <type_traits>

#include "szx_device.cuh"
#include "szx_launch.h"

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
    uint64_t total_bytes;
    uint64_t copy_ns;    // wall-time limit of the record copy wait
    uint64_t rows_full;  // 128-byte output rows fully inside the output
    uint32_t use_tma;    // store full rows with the tensor store (else plain stores)
};

__device__ __forceinline__ void flag_status(uint32_t *status, uint32_t code) {
    if (status) atomicMax(status, code);
}

__device__ __forceinline__ uint32_t dprmt(uint32_t a, uint32_t b, uint32_t s) { return __byte_perm(a, b, s); }

// Tables (compile time), per plane j in 0..2 and the 2-bit codes of four
// values (value k at bits 2k):
//   expand: byte-permute selector moving the k-th byte of a run to the k-th
//           value whose code is <= j (others get zero) | count << 16;
//   carry:  byte-permute selector for the copy-forward of plane j: a value
//           whose code is > j takes the byte of the nearest earlier value of
//           the group with code <= j, or the carry byte (operand byte 4).
struct DecodeLut {
    uint32_t expand[768];
    uint32_t carry[768];
};
constexpr DecodeLut make_decode_lut() {
    DecodeLut t{};
    for (uint32_t i = 0; i < 768; ++i) {
        const uint32_t j = i >> 8, code = i & 255u;
        uint32_t sel = 0x4444u, cnt = 0, csel = 0;
        int src = -1;
        for (uint32_t k = 0; k < 4; ++k) {
            const bool own = ((code >> (2 * k)) & 3u) <= j;
            if (own) {
                sel = (sel & ~(0xFu << (4 * k))) | (cnt << (4 * k));
                ++cnt;
                src = (int)k;
            }
            csel |= (uint32_t)(src < 0 ? 4 : src) << (4 * k);
        }
        t.expand[i] = sel | (cnt << 16);
        t.carry[i] = csel;
    }
    return t;
}
__device__ const DecodeLut kDecodeLut = make_decode_lut();

__device__ __forceinline__ void transpose4d(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, uint32_t (&W)[4]) {
    const uint32_t a = dprmt(t0, t1, 0x5140), b = dprmt(t0, t1, 0x7362);
    const uint32_t c = dprmt(t2, t3, 0x5140), d = dprmt(t2, t3, 0x7362);
    W[3] = dprmt(a, c, 0x5410);
    W[2] = dprmt(a, c, 0x7632);
    W[1] = dprmt(b, d, 0x5410);
    W[0] = dprmt(b, d, 0x7632);
}

// The up to 4 bytes at byte offset p of a shared-memory byte buffer (with 8
// bytes of readable slack after its end), little-endian.
__device__ __forceinline__ uint32_t load_run(const uint8_t *buf, uint32_t p) {
    const uint32_t *wp = reinterpret_cast<const uint32_t *>(buf) + (p >> 2);
    return __funnelshift_r(wp[0], wp[1], (p & 3u) * 8u);
}

constexpr int kDStages = 3;
constexpr int kDConsumers = kThreads;                 // 8 decoding warps
constexpr int kDProducerWarp = kDConsumers / 32;      // warp 8
constexpr int kDStorerWarp = kDProducerWarp + 1;      // warp 9
constexpr int kDThreads = kDConsumers + 64;
constexpr uint32_t kBitsWindow = 64;  // 16-byte-aligned window holding a tile's state bits

// Per stage (1024-byte aligned, for the swizzled tensor store): the buffer
// that receives the record and then holds the decoded tile, the tile's mu
// values, its state-bit window and its blocks' mid-byte counts.
struct DSmem {
    uint32_t stage;          // stage stride; stage st starts at st * stage
    uint32_t mu, bits, mk;   // offsets inside a stage (the buffer is at 0)
    uint32_t lut, total;
};
__host__ __device__ inline DSmem decompress_smem(uint32_t G, uint32_t b, uint32_t w) {
    DSmem s;
    const uint32_t tile = G * b * w;
    const uint32_t rec = record_max_bytes(G, b, w) + 16;  // + slack for the 8-byte run reads
    const uint32_t body = ((tile > rec ? tile : rec) + 15) & ~15u;
    const uint32_t mub = (G * w + 15) & ~15u;
    s.stage = (body + mub + kBitsWindow + 4 * G + 1023) & ~1023u;
    s.mu = body;
    s.bits = s.mu + mub;
    s.mk = s.bits + kBitsWindow;
    s.lut = kDStages * s.stage;
    s.total = s.lut + (uint32_t)sizeof(DecodeLut) + 1024;  // + slack to realign the dynamic base
    return s;
}

__device__ __forceinline__ void decoder_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kDConsumers) : "memory"); }

__device__ __forceinline__ void dmbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

// Persistent decoder: tile = blockIdx.x + k * gridDim.x.
template <typename T, int LPB, int VPL>
__global__ void __launch_bounds__(kDThreads, (VPL * sizeof(T) > 128) ? 1 : 2)
    decompress_kernel(const __grid_constant__ CUtensorMap tmap, DecompressArgs a) {
    using F = Fmt<T>;
    using U = typename F::U;
    constexpr int w = F::w;
    constexpr int W = F::W;
    constexpr int BPW = 32 / LPB;
    constexpr int NCODE = (2 * VPL + 31) / 32;
    constexpr int NPW = W / 32;         // 32-bit words per value
    constexpr int RPL = VPL * w / 128;  // 128-byte rows per lane
    static_assert(RPL >= 1, "lane geometry");

    extern __shared__ __align__(16) uint8_t smem_raw[];  // realigned to 1024 below
    // full: record, mu and state bits copied in; done: tile decoded into the
    // stage; empty: tile stored, stage free
    __shared__ __align__(8) uint64_t full[kDStages], done[kDStages], empty[kDStages];
    // st_bad: set by the producer (index or header fault); st_dbad: set by a
    // decoder (bad codes), read only after the first barrier
    __shared__ uint32_t st_tile[kDStages], st_size[kDStages], st_bad[kDStages], st_dbad[kDStages],
        st_boff[kDStages], st_store[kDStages];
    __shared__ uint32_t s_abort;

    uint8_t *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const Geometry &g = a.g;
    const uint32_t b = g.b, G = g.G;
    const DSmem L = decompress_smem(G, b, w);
    const DecodeLut *lut = reinterpret_cast<const DecodeLut *>(smem + L.lut);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr uint32_t kNone = 0xFFFFFFFFu;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(&kDecodeLut);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + L.lut);
        for (uint32_t i = tid; i < sizeof(DecodeLut) / 16; i += kDThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int i = 0; i < kDStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&done[i], kDConsumers / 32);
            mbar_init(&empty[i], 1);
            st_tile[i] = kNone;
            st_size[i] = st_bad[i] = st_dbad[i] = st_boff[i] = st_store[i] = 0;
        }
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    if (warp == kDProducerWarp) {
        // ---- producer: record, mu and state-bit copies into the ring --------
        if (lane != 0) return;
        const uint32_t rec_max = record_max_bytes(G, b, w);
        const uint64_t *idx = reinterpret_cast<const uint64_t *>(a.in + g.off_index);
        // per stage (bit st): is its last phase a copy (then it may still be in
        // flight when the producer is done), and that phase's parity
        uint32_t copy_last = 0, copy_par = 0;
        uint64_t n0 = 0, n1 = 0;  // index entries of the next tile
        if (blockIdx.x < g.ntiles) {
            n0 = idx[blockIdx.x];
            n1 = idx[blockIdx.x + 1];
        }
        for (uint32_t it = 0;; ++it) {
            const int st = (int)(it % kDStages);
            const uint32_t k = it / kDStages;
            const uint64_t tile64 = (uint64_t)blockIdx.x + (uint64_t)it * gridDim.x;
            const uint32_t tile = tile64 < g.ntiles ? (uint32_t)tile64 : kNone;
            const uint64_t r0 = n0, r1 = n1;
            // load the following tile's entries now; they arrive while this
            // iteration waits for its stage
            const uint64_t next = tile64 + gridDim.x;
            if (next < g.ntiles) {
                n0 = idx[next];
                n1 = idx[next + 1];
            }
            if (it >= kDStages && !mbar_wait_bounded(&empty[st], (k - 1) & 1u, 8 * a.copy_ns)) {
                flag_status(a.status, 6u);
                break;
            }
            uint32_t bad = 0, size = 0;
            if (tile != kNone) {
                if (a.check_header && tile == 0) {
                    const uint32_t *h32 = reinterpret_cast<const uint32_t *>(a.in);
                    const uint64_t *h64 = reinterpret_cast<const uint64_t *>(a.in);
                    if (h32[0] != kMagic || (h32[1] & 0xFFFFu) != (kVersion | (a.dtype << 8)) || h32[2] != b ||
                        h32[3] != G || h64[2] != g.n || h64[7] != a.total_bytes)
                        bad = 1;
                }
                if (r0 > r1 || r1 > a.rec_total || (r0 & 15) || (r1 & 15) || r1 - r0 > rec_max) bad = 1;
                if (tile == g.ntiles - 1 && r1 != a.rec_total) bad = 1;
                size = bad ? 0u : (uint32_t)(r1 - r0);
            }
            st_tile[st] = tile;
            st_size[st] = size;
            st_bad[st] = bad;
            st_dbad[st] = 0;
            if (tile != kNone && !bad) {
                const uint64_t k0 = (uint64_t)tile * G;
                const uint32_t Gt = (uint32_t)min_u64(G, g.nb - k0);
                // mu values: G * w is a multiple of 32, and the section is
                // padded to 16 bytes, so the rounded copy stays inside it
                const uint32_t mu_bytes = (uint32_t)pad16((uint64_t)Gt * w);
                // state bits: the 16-byte-aligned window around the tile's bytes
                const uint64_t sb0 = g.off_state + k0 / 8;
                const uint64_t sbA = sb0 & ~uint64_t(15);
                const uint64_t sbE = pad16(g.off_state + (k0 + Gt + 7) / 8);
                st_boff[st] = (uint32_t)(sb0 - sbA);
                mbar_arrive_expect_tx(&full[st], size + mu_bytes + (uint32_t)(sbE - sbA));
                if (size) bulk_g2s(smem + st * L.stage, a.in + g.off_rec + r0, size, &full[st]);
                bulk_g2s(smem + st * L.stage + L.mu, a.in + g.off_mu + k0 * w, mu_bytes, &full[st]);
                bulk_g2s(smem + st * L.stage + L.bits, a.in + sbA, (uint32_t)(sbE - sbA), &full[st]);
                copy_last |= 1u << st;
                copy_par = (copy_par & ~(1u << st)) | ((k & 1u) << st);
            } else {
                dmbar_arrive(&full[st]);
                copy_last &= ~(1u << st);
            }
            if (tile == kNone) break;
        }
        // do not leave while a copy may still be writing into shared memory
        for (int st = 0; st < kDStages; ++st)
            if ((copy_last >> st) & 1u) mbar_wait_bounded(&full[st], (copy_par >> st) & 1u, a.copy_ns);
        return;
    }

    if (warp == kDStorerWarp) {
        // ---- storer: tensor stores of decoded tiles ------------------------
        if (lane != 0) return;
        for (uint32_t it = 0;; ++it) {
            const int st = (int)(it % kDStages);
            const uint32_t k = it / kDStages;
            if (!mbar_wait_bounded(&done[st], k & 1u, 8 * a.copy_ns)) {
                flag_status(a.status, 6u);
                break;
            }
            const uint32_t tile = st_tile[st];
            if (tile >= g.ntiles) break;
            const uint64_t row0 = (uint64_t)tile * 256 * RPL;
            if (st_store[st] && a.use_tma && row0 < a.rows_full) {
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    const uint64_t y = row0 + 256 * (uint64_t)i;
                    if (y < a.rows_full) {
                        asm volatile(
                            "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                                reinterpret_cast<uint64_t>(&tmap)),
                            "r"(0), "r"((int)y), "r"(smem_addr(smem + st * L.stage + i * 32768))
                            : "memory");
                    }
                }
                bulk_commit();
                bulk_wait_read_all();  // the stage may be refilled once the store has read it
            }
            dmbar_arrive(&empty[st]);
        }
        bulk_wait_all();
        return;
    }

    // ---- decoders (warps 0..7) ---------------------------------------------
    for (uint32_t it = 0;; ++it) {
        const int st = (int)(it % kDStages);
        const uint32_t k = it / kDStages;
        if (!mbar_wait_bounded(&full[st], k & 1u, a.copy_ns)) s_abort = 1;
        const uint32_t tile = st_tile[st];
        const uint32_t size = st_size[st];
        uint8_t *rec = smem + st * L.stage;
        uint32_t *sm_mk = reinterpret_cast<uint32_t *>(smem + st * L.stage + L.mk);
        const uint64_t k0 = (uint64_t)tile * G;
        const uint32_t Gt = tile < g.ntiles ? (uint32_t)min_u64(G, g.nb - k0) : 0u;

        // ---- ranks, codes, mid-byte counts --------------------------------
        const int sub = lane % LPB;
        const uint32_t blk = (uint32_t)(warp * BPW + lane / LPB);
        const bool exists = blk < Gt && !st_bad[st];
        const uint64_t kg = k0 + blk;
        const int len = exists ? (int)min_u64(b, g.n - kg * b) : 0;
        int nvalid = len - sub * VPL;
        nvalid = nvalid < 0 ? 0 : (nvalid > VPL ? VPL : nvalid);
        const bool full_lane = nvalid == VPL;
        // rank of the block among the tile's non-constant blocks: a popcount
        // of the tile's state bits below it (the tile's bits start at a byte)
        uint32_t rank = 0;
        bool nonconst = false;
        uint32_t nn_t = 0;
        if (tile < g.ntiles && !st_bad[st]) {
            const uint8_t *stb = smem + st * L.stage + L.bits + st_boff[st];
            for (uint32_t i = 0; i < (Gt + 7) / 8; i += 4) {
                uint32_t wv = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i + j < (Gt + 7) / 8) wv |= (uint32_t)stb[i + j] << (8 * j);
                const uint32_t base = i * 8;
                if (Gt - base < 32) wv &= (1u << (Gt - base)) - 1u;
                nn_t += __popc(wv);
                if (exists && blk >= base) {
                    if (blk < base + 32) {
                        rank += __popc(wv & ((1u << (blk - base)) - 1u));
                        nonconst = (wv >> (blk - base)) & 1u;
                    } else {
                        rank += __popc(wv);
                    }
                }
            }
        }
        bool ok = (uint64_t)nn_t * (b / 4 + 1) <= size;
        nonconst = nonconst && ok;
        const int rq = nonconst ? (int)rec[nn_t * (b / 4) + rank] : 0;
        const bool raw = nonconst && rq == 0xFF;
        const bool coded = nonconst && !raw;
        if (coded && !(rq >= 1 + F::E && rq <= W)) ok = false;
        const int s = (8 - (rq & 7)) & 7;
        const int q = coded && ok ? (rq + s) >> 3 : 2;
        const int lmax = q < 3 ? q : 3;
        uint32_t codes[NCODE];
#pragma unroll
        for (int i = 0; i < NCODE; ++i) codes[i] = 0;
        if (coded && ok) {
            const uint8_t *lead = rec + rank * (b / 4) + sub * (VPL / 4);
            if constexpr (NCODE == 2) {
                const uint2 v = *reinterpret_cast<const uint2 *>(lead);
                codes[0] = v.x;
                codes[1] = v.y;
            } else {
                codes[0] = *reinterpret_cast<const uint32_t *>(lead);
            }
            // codes past the end are 0; no code exceeds min(3, q)
#pragma unroll
            for (int i = 0; i < NCODE; ++i) {
                const int nv = nvalid - 16 * i;
                const uint32_t vm = nv >= 16 ? 0xFFFFFFFFu : (nv <= 0 ? 0u : (0xFFFFFFFFu >> (2 * (16 - nv))));
                if (codes[i] & ~vm) ok = false;
                if (lmax == 2 && (codes[i] & (codes[i] >> 1) & 0x55555555u)) ok = false;
            }
        }
        uint32_t suml = 0;
#pragma unroll
        for (int i = 0; i < NCODE; ++i) suml += __popc(codes[i] & 0x55555555u) + 2 * __popc(codes[i] & 0xAAAAAAAAu);
        uint32_t mk = coded ? (uint32_t)(nvalid * q) - suml : (raw ? (uint32_t)nvalid * w : 0u);
        const uint32_t segmask = (LPB == 32 ? kFull : ((1u << LPB) - 1u)) << (lane & ~(LPB - 1));
        {
            const uint32_t bal = __ballot_sync(kFull, ok);
            ok = (bal & segmask) == segmask;
        }
#pragma unroll
        for (int d = 1; d < LPB; d <<= 1) mk += __shfl_xor_sync(kFull, mk, d);
        if (blk < G && sub == 0) sm_mk[blk] = (exists && nonconst) ? mk : 0u;
        if (!ok && exists) st_dbad[st] = 1;
        decoder_sync();
        if (s_abort || tile >= g.ntiles) {
            // hand the stage to the storer (it stops on the same tile), and stop
            if (tid == 0) st_tile[st] = kNone;
            decoder_sync();
            if (lane == 0) dmbar_arrive(&done[st]);
            break;
        }

        // ---- mid-byte offsets: every warp scans the tile's counts ----------
        uint32_t midoff, total;
        {
            const uint32_t per = (Gt + 31) / 32;
            const uint32_t lo = min(lane * per, Gt), hi = min(lo + per, Gt);
            uint32_t c = 0;
            for (uint32_t kk = lo; kk < hi; ++kk) c += sm_mk[kk];
            uint32_t e = warp_exclusive_scan(c, &total);
            const uint32_t chunk = blk / (per ? per : 1u);
            uint32_t before = __shfl_sync(kFull, e, chunk < 32 ? (int)chunk : 0);
            for (uint32_t kk = chunk * per; kk < blk && kk < Gt; ++kk) before += sm_mk[kk];
            midoff = before;
        }
        const uint32_t used = nn_t * (b / 4 + 1) + total;
        // uniform over the CTA: st_bad and the counts were fixed before the barrier
        const bool bad = st_bad[st] || st_dbad[st] || pad16(used) != size;
        U x[VPL];
        if (bad) {
            if (tid == 0) flag_status(a.status, 3u);
        } else {
            // ---- decode --------------------------------------------------
            const uint32_t mbase = nn_t * (b / 4 + 1) + midoff;
            const U mu_bits = exists ? reinterpret_cast<const U *>(smem + st * L.stage + L.mu)[blk] : U(0);

            using CntT = std::conditional_t<(LPB * VPL > 1023), unsigned long long, uint32_t>;
            constexpr int FB = LPB * VPL > 1023 ? 16 : 10;
            constexpr CntT FM = (CntT(1) << FB) - 1;
            CntT cnt = 0;
            if (coded) {
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
            const uint32_t n0 = (uint32_t)(tot & FM), n1 = (uint32_t)((tot >> FB) & FM),
                           n2 = (uint32_t)((tot >> (2 * FB)) & FM);
            const uint32_t cj[3] = {(uint32_t)(cnt & FM), (uint32_t)((cnt >> FB) & FM),
                                    (uint32_t)((cnt >> (2 * FB)) & FM)};
            uint32_t pos0 = mbase + (uint32_t)(off & FM);
            uint32_t pos1 = mbase + n0 + (uint32_t)((off >> FB) & FM);
            uint32_t pos2 = mbase + n0 + n1 + (uint32_t)((off >> (2 * FB)) & FM);
            const uint32_t dense0 = mbase + n0 + n1 + n2 + (uint32_t)sub * VPL;

            // carries into the lane for the planes that can inherit (j < lmax):
            // the last own byte of the nearest lower lane of the block that owns one
            uint32_t carry[3];
            {
                const uint32_t below = segmask & ((1u << lane) - 1u);
                const uint32_t pj[3] = {pos0, pos1, pos2};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const bool has = coded && j < lmax && cj[j] > 0;
                    const uint32_t last = has ? rec[pj[j] + cj[j] - 1] : 0u;
                    const uint32_t m = __ballot_sync(kFull, has) & below;
                    const uint32_t v = __shfl_sync(kFull, last, m ? 31 - __clz(m) : 0);
                    carry[j] = m ? v : 0u;
                }
            }

            if (coded) {
                const T mu = F::from(mu_bits);
#pragma unroll
                for (int gq = 0; gq < VPL / 4; ++gq) {
                    uint32_t code8 = (codes[gq >> 2] >> (8 * (gq & 3))) & 0xFFu;
                    uint32_t dense8 = 0;
                    if (!full_lane) {
                        const int nv = nvalid - 4 * gq;
                        const uint32_t inval = nv >= 4 ? 0u : (nv <= 0 ? 0xFFu : (0xFFu << (2 * nv)) & 0xFFu);
                        code8 |= inval;
                        dense8 = inval;
                    }
                    // plane words: byte k = byte j of value 4gq + k
                    uint32_t P[W / 8];
#pragma unroll
                    for (int j = 0; j < W / 8; ++j) P[j] = 0;
                    {
                        const uint32_t e0 = lut->expand[code8];
                        P[0] = dprmt(load_run(rec, pos0), 0, e0);
                        pos0 += e0 >> 16;
                        const uint32_t e1 = lut->expand[256 + code8];
                        P[1] = dprmt(load_run(rec, pos1), 0, e1);
                        pos1 += e1 >> 16;
                        if (q >= 3) {
                            const uint32_t e2 = lut->expand[512 + code8];
                            P[2] = dprmt(load_run(rec, pos2), 0, e2);
                            pos2 += e2 >> 16;
                        }
                        if (q >= 4) {
                            const uint32_t sel = full_lane ? 0x3210u : lut->expand[512 + dense8];
#pragma unroll
                            for (int j = 3; j < W / 8; ++j)
                                if (j < q)
                                    P[j] = dprmt(load_run(rec, dense0 + (uint32_t)(j - 3) * len + 4 * gq), 0, sel);
                        }
                    }
                    // leading bytes: copy the nearest earlier owner forward
                    P[0] = dprmt(P[0], carry[0], lut->carry[code8]);
                    carry[0] = P[0] >> 24;
                    P[1] = dprmt(P[1], carry[1], lut->carry[256 + code8]);
                    carry[1] = P[1] >> 24;
                    if (lmax >= 3) {
                        P[2] = dprmt(P[2], carry[2], lut->carry[512 + code8]);
                        carry[2] = P[2] >> 24;
                    }
                    // planes back to words: t = (P0.k, P1.k, P2.k, P3.k), most significant first
                    U t[4];
                    if constexpr (NPW == 1) {
                        uint32_t Wq[4];
                        transpose4d(P[3], P[2], P[1], P[0], Wq);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) t[kk] = Wq[3 - kk];
                    } else {
                        uint32_t Wh[4], Wl[4];
                        transpose4d(P[3], P[2], P[1], P[0], Wh);
                        transpose4d(P[7], P[6], P[5], P[4], Wl);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) t[kk] = ((U)Wh[3 - kk] << 32) | (U)Wl[3 - kk];
                    }
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) x[4 * gq + kk] = F::bits(F::add(F::from((U)(t[kk] << s)), mu));
                }
            } else if (raw) {
                const uint8_t *p = rec + mbase + (uint32_t)sub * VPL * w;
#pragma unroll
                for (int m = 0; m < VPL; ++m) {
                    U u = 0;
                    if (m < nvalid) {
#pragma unroll
                        for (int i = 0; i < w; ++i) u |= (U)p[m * w + i] << (8 * i);
                    }
                    x[m] = u;
                }
            } else {
#pragma unroll
                for (int m = 0; m < VPL; ++m) x[m] = mu_bits;
            }

            // strictness: the record's pad bytes must be zero
            if (warp == 0)
                for (uint32_t i = used + lane; i < size; i += 32)
                    if (rec[i]) flag_status(a.status, 3u);
        }
        decoder_sync();  // the record is no longer read: the stage takes the output

        if (!bad) {
            if (exists && nvalid > 0) {
                const uint32_t lane_row0 = (uint32_t)((warp * 32 + lane) * RPL);
                const uint64_t grow0 = (uint64_t)tile * 256 * RPL + lane_row0;
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) {
                    constexpr int VPR = 128 / w;  // values per row
                    const int nv = nvalid - rr * VPR;
                    if (nv <= 0) continue;
                    if (a.use_tma && grow0 + rr < a.rows_full) {
                        // full row: 128-byte-swizzled into the stage for the tensor store
                        const uint32_t rowi = lane_row0 + rr;
                        uint8_t *row = smem + st * L.stage + (rowi << 7);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            uint4 v;
                            U *u = reinterpret_cast<U *>(&v);
#pragma unroll
                            for (int kk = 0; kk < 16 / w; ++kk) u[kk] = x[rr * VPR + c * (16 / w) + kk];
                            *reinterpret_cast<uint4 *>(row + ((c ^ (rowi & 7u)) << 4)) = v;
                        }
                    } else {
                        U *dst = reinterpret_cast<U *>(a.out) + kg * b + sub * VPL + rr * VPR;
                        if (nv >= VPR) {
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                uint4 v;
                                U *u = reinterpret_cast<U *>(&v);
#pragma unroll
                                for (int kk = 0; kk < 16 / w; ++kk) u[kk] = x[rr * VPR + c * (16 / w) + kk];
                                reinterpret_cast<uint4 *>(dst)[c] = v;
                            }
                        } else {
#pragma unroll
                            for (int m = 0; m < VPR; ++m)
                                if (m < nv) dst[m] = x[rr * VPR + m];
                        }
                    }
                }
            }
        }
        if (tid == 0) st_store[st] = bad ? 0u : 1u;
        // the storer takes the stage once every warp has written its rows
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) dmbar_arrive(&done[st]);
    }
}

// ---------------------------------------------------------------------------

template <typename T, int LPB, int VPL>
static cudaError_t launch_t(const CUtensorMap &tm, const DecompressArgs &a, cudaStream_t stream) {
    const DSmem L = decompress_smem(a.g.G, a.g.b, Fmt<T>::w);
    auto kern = decompress_kernel<T, LPB, VPL>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0, per_sm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDThreads, L.total)) != cudaSuccess)
        return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint64_t grid = min_u64(a.g.ntiles, (uint64_t)sms * per_sm);
    kern<<<(unsigned)grid, kDThreads, L.total, stream>>>(tm, a);
    return cudaGetLastError();
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
    a.rows_full = n * (dtype == 0 ? 4 : 8) / 128;
    CUtensorMap tm;
    a.use_tma = encode_row_map(&tm, out, a.rows_full) ? 1u : 0u;
    if (dtype == 0) {
        switch (block) {
            case 32: return launch_t<float, 1, 32>(tm, a, stream);
            case 64: return launch_t<float, 2, 32>(tm, a, stream);
            case 128: return launch_t<float, 4, 32>(tm, a, stream);
            case 256: return launch_t<float, 8, 32>(tm, a, stream);
            case 512: return launch_t<float, 16, 32>(tm, a, stream);
            case 1024: return launch_t<float, 32, 32>(tm, a, stream);
        }
    } else {
        switch (block) {
            case 32: return launch_t<double, 2, 16>(tm, a, stream);
            case 64: return launch_t<double, 4, 16>(tm, a, stream);
            case 128: return launch_t<double, 8, 16>(tm, a, stream);
            case 256: return launch_t<double, 16, 16>(tm, a, stream);
            case 512: return launch_t<double, 32, 16>(tm, a, stream);
            case 1024: return launch_t<double, 32, 32>(tm, a, stream);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace szx
