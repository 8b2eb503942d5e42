// decompress.cu -- SZx decompression kernel for sm_103a.
//
// Persistent CTAs decode tiles of G blocks.  The tile index written by the
// compressor gives each record's offset, so tiles decode independently: no
// device-wide scan is left for decompression (the paper's GPU decoder, Sec.
// V-B, runs a prefix scan of the mid-byte counts first).  Per CTA, a producer
// thread, an indexing warp and eight decoding warps share up to six tiles in
// flight through mbarriers per tile slot (head / full / indexed / consumed):
//   producer (one thread): per tile, bulk-copies (cp.async.bulk) the record
//     into a shared-memory ring, where it takes its own size, and the tile's
//     mu values and a 16-byte-aligned window of its state bits into the
//     tile's slot; it frees ring space in tile order as the decoders release
//     tiles.  The record's head (reqBits bytes and lead codes), the mu
//     values and the state bits complete one mbarrier and the rest of the
//     record another, so that indexing starts before the mid bytes have
//     landed.  The tile index entries are loaded one tile ahead, so no global
//     latency sits between two copies;
//   indexing warp: per tile, ranks every block among the tile's non-constant
//     blocks (a popcount of the state bits), reads its reqBits byte and lead
//     codes, checks them, counts its mid bytes, and scans the counts into
//     each block's mid-byte offset; the total is checked against the record
//     size, so that every later read is inside the record.  It writes a
//     block table (offset, rank, reqBits) and the tile's verdict, ahead of
//     the decoders;
//   eight decoding warps: decode the tile's record into registers, release
//     the tile, then write their rows into a buffer of their own in the
//     128-byte-swizzled layout of the TMA tensor store and issue that store
//     (one 2-D box of 32 rows per warp).  The ragged last row goes out with
//     plain stores.  Warp 0 also checks that the record's padding is zero.
// The same kernel serves a single stream (its descriptor is a kernel
// parameter; CTA c takes tiles c, c + gridDim.x, ...) and batches (a table
// of descriptors in device memory, BATCH; CTAs take tiles by ticket, which
// balances fields of unequal cost), and decodes a block range for random
// access.  Tiles wholly inside the field and the range run a copy of the
// decoders' work compiled for full blocks.
//
// Work layout as in the compressor: every lane owns 128 contiguous output
// bytes (32 f32 or 16 f64 values); a block of b values spans LPB = b / VPL
// adjacent lanes.  Every lane reads its block's table entry and its own lead
// codes and rebuilds its values: for each group of four values and each byte
// plane, the lane's run of own bytes is read with two aligned word loads and
// a funnel shift, and one table-driven byte permute both spreads it to the
// owning values and copies a leading byte (identical to the previous
// value's) forward from the nearest earlier owner, or from the carry into
// the lane -- the last own byte of the nearest lower lane of the block that
// owns one (a ballot and a shuffle).  This is the paper's index propagation
// (Sec. V-B) in one step per plane.  When every lane of a warp owns byte 2
// of all its values, plane 2 needs neither: each group's word is a funnel
// shift of two consecutive words of the run.  A byte transpose turns planes
// back into words; then v' = t << s and d' = RN(v' + mu).
#include <cstring>
#include <type_traits>

#include "szx_device.cuh"
#include "szx_launch.h"

namespace szx {

struct DecompressLaunch {
    const DField *fields;  // device table of nfields fields, or null: the single field
    uint32_t nfields;
    uint64_t total_tiles;  // tiles of all fields, field after field
    uint64_t copy_ns;      // wall-time limit of a copy wait
    // batches: tile tickets (zeroed before the launch), CTAs take tiles as
    // they go; a single stream: null, CTA c takes tiles c, c + gridDim.x, ...
    uint32_t *ticket;
};

template <bool BATCH>
__device__ __forceinline__ const DField *dfield_ptr(const DField &one, const DecompressLaunch &lc, uint32_t f) {
    if constexpr (BATCH) return lc.fields + f;
    else return &one;  // the kernel parameter itself (param space)
}

// The field holding global tile t: the last one whose first tile is <= t.
template <bool BATCH>
__device__ __forceinline__ uint32_t dfield_of(const DecompressLaunch &lc, uint64_t t) {
    if constexpr (!BATCH) return 0;
    uint32_t lo = 0, hi = lc.nfields - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (lc.fields[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void flag_status(uint32_t *status, uint32_t code) {
    if (status) atomicMax(status, code);
}

__device__ __forceinline__ uint32_t dprmt(uint32_t a, uint32_t b, uint32_t s) { return __byte_perm(a, b, s); }

// Table (compile time), per plane j in 0..2 and the 2-bit codes of four values
// (value k at bits 2k): a byte-permute selector that, applied to (run of own
// bytes, carry byte), gives value k the next byte of the run if it owns one
// (code <= j), else the byte of the nearest earlier owner of the group, else
// the carry byte (operand byte 4) -- expansion and the copy-forward of
// identical leading bytes in one permute -- plus the number of owners << 16.
struct DecodeLut {
    uint32_t sel[768];
};
constexpr DecodeLut make_decode_lut() {
    DecodeLut t{};
    for (uint32_t i = 0; i < 768; ++i) {
        const uint32_t j = i >> 8, code = i & 255u;
        uint32_t sel = 0, cnt = 0;
        int last = -1;
        for (uint32_t k = 0; k < 4; ++k) {
            const bool own = ((code >> (2 * k)) & 3u) <= j;
            uint32_t nib = 0;
            if (own) {
                nib = cnt;
                last = (int)cnt;
                ++cnt;
            } else {
                nib = last < 0 ? 4u : (uint32_t)last;
            }
            sel |= nib << (4 * k);
        }
        t.sel[i] = sel | (cnt << 16);
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

constexpr int kDSlots = 6;  // tiles in flight per CTA, at most (their records share one ring)
// A CTA has NDW decoding warps (8 or 4), then the producer and the indexing
// warp; each decoding lane rebuilds RPL = rows / (32 NDW) consecutive 128-byte
// rows of the tile.
__host__ __device__ constexpr int decompress_threads(int ndw) { return ndw * 32 + 64; }
constexpr uint32_t kBitsWindow = 64;  // 16-byte-aligned window holding a tile's state bits

// Shared memory: one output buffer per decoding warp (its 32 * RPL rows of
// 128 bytes, 1024-byte aligned for the swizzled tensor store), the decode
// table, kDSlots tile slots (each: the tile's mu values, its state-bit window
// and its block table), and the record ring, which takes the rest of the
// CTA's share of the SM (two CTAs per SM for 32 KiB tiles, one for 64 KiB).
// Records sit in the ring at their own size, so that at a typical ratio four
// or five tiles are in flight, and at worst (every block raw) two.
struct DSmem {
    uint32_t wbuf, wbuf_bytes;  // warp w's output buffer at wbuf + w * wbuf_bytes
    uint32_t lut;
    uint32_t slots, slot;       // slot i at slots + i * slot
    uint32_t mu, bits, info;    // offsets inside a slot
    uint32_t ring, ring_bytes;  // the record ring (128-aligned, a multiple of 1024 bytes)
    uint32_t total;
};
__host__ __device__ inline DSmem decompress_smem(uint32_t G, uint32_t b, uint32_t w, uint32_t ndw) {
    DSmem s;
    const uint32_t tile = G * b * w;  // 32 KiB, or 64 KiB for f64 with b = 1024
    // (the per-CTA limit includes the static barriers and slot words)
    const uint32_t budget = tile > 32768u ? 226u * 1024u : 112u * 1024u;
    constexpr uint32_t kRealign = 1024;  // slack to realign the dynamic base to 1024
    s.wbuf = 0;
    s.wbuf_bytes = tile / ndw;  // 4 KiB per 128-byte row per lane
    s.lut = s.wbuf + tile;
    s.slots = s.lut + (uint32_t)sizeof(DecodeLut);
    s.mu = 0;
    s.bits = (G * w + 15) & ~15u;
    s.info = s.bits + kBitsWindow;
    s.slot = s.info + ((8 * G + 15) & ~15u);
    s.ring = (s.slots + kDSlots * s.slot + 127) & ~127u;
    s.ring_bytes = (budget - kRealign - s.ring) & ~1023u;
    s.total = s.ring + s.ring_bytes + kRealign;
    return s;
}

__device__ __forceinline__ void dmbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

// Persistent decoder: tile = blockIdx.x + it * gridDim.x for it = 0, 1, ...
template <typename T, int LPB, int VPL, int NDW, bool BATCH>
__global__ void __launch_bounds__(decompress_threads(NDW),
                                  (tile_blocks(LPB * VPL, sizeof(T)) * LPB * VPL * sizeof(T) > 32768) ? 1 : 2)
    decompress_kernel(const __grid_constant__ DField one, const __grid_constant__ DecompressLaunch lc) {
    constexpr int kDWarps = NDW;
    constexpr int kDThreads = decompress_threads(NDW);
    constexpr int kDProducerWarp = NDW;
    constexpr int kDIndexerWarp = NDW + 1;
    using F = Fmt<T>;
    using U = typename F::U;
    constexpr int w = F::w;
    constexpr int W = F::W;
    constexpr int BPW = 32 / LPB;
    constexpr int NCODE = (2 * VPL + 31) / 32;
    constexpr int NPW = W / 32;         // 32-bit words per value
    constexpr int RPL = VPL * w / 128;  // 128-byte rows per lane
    constexpr uint32_t b = (uint32_t)(LPB * VPL);
    constexpr uint32_t G = tile_blocks(b, (uint32_t)w);
    constexpr uint32_t TILE_ROWS = G * b * w / 128;  // 256, or 512 for 64 KiB tiles
    static_assert(RPL >= 1 && (uint32_t)(NDW * 32 * RPL) == TILE_ROWS, "lane geometry");
    // output boxes of the row map: 32 rows, or 64 for the 64 KiB tiles of 8 warps
    constexpr uint32_t BOX_ROWS = TILE_ROWS / 8;
    constexpr uint32_t WARP_BOXES = 32u * RPL / BOX_ROWS;
    constexpr uint32_t kHeadBytes = (G * (b / 4 + 1) + 15) & ~15u;  // reqBits bytes and lead codes, at most

    extern __shared__ __align__(16) uint8_t smem_raw[];  // realigned to 1024 below
    // head: the record's head (reqBits bytes and lead codes), mu values and
    // state bits copied in; full: the rest of the record; indexed: the
    // indexing warp has written the tile's block table and verdict;
    // consumed: every decoding warp is done with the tile (record and slot)
    __shared__ __align__(8) uint64_t head[kDSlots], full[kDSlots], indexed[kDSlots], consumed[kDSlots];
    // st_bad: set by the producer (index or header fault); st_verdict: set by
    // the indexing warp (0: decode, 3: corrupt record, 6: a wait ran out)
    __shared__ uint32_t st_size[kDSlots], st_bad[kDSlots], st_verdict[kDSlots], st_boff[kDSlots];
    __shared__ uint32_t st_used[kDSlots];  // the record's bytes before its zero padding (when the verdict is 0)
    __shared__ uint32_t st_field[kDSlots], st_tile[kDSlots];  // the slot's field and its local tile
    __shared__ uint32_t st_off[kDSlots];                       // the slot's record: offset in the ring
    __shared__ __align__(8) unsigned long long st_end[kDSlots];  // its end, as a position of the ring's sequence

    uint8_t *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const DSmem L = decompress_smem(G, b, w, NDW);
    const uint32_t *lut = reinterpret_cast<const uint32_t *>(smem + L.lut);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(&kDecodeLut);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + L.lut);
        for (uint32_t i = tid; i < sizeof(DecodeLut) / 16; i += kDThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int i = 0; i < kDSlots; ++i) {
            mbar_init(&head[i], 1);
            mbar_init(&full[i], 1);
            mbar_init(&indexed[i], 1);
            mbar_init(&consumed[i], kDWarps);
            st_size[i] = st_bad[i] = st_verdict[i] = st_boff[i] = st_used[i] = st_field[i] = st_tile[i] = st_off[i] = 0;
            st_end[i] = 0;
        }
        fence_mbar_init();
    }
    __syncthreads();
    // nothing above reads or writes memory that an earlier kernel may write
    // (the launch may be the programmatic dependent of the status clear)
    wait_prior_grids();

    if (warp == kDProducerWarp) {
        // ---- producer: record copies into the ring, mu and state bits into the slots
        if (lane != 0) return;
        const uint32_t rec_max = record_max_bytes(G, b, w);
        // per slot (bit st): is its last phase a copy (then it may still be in
        // flight when the producer is done), and that phase's parity
        uint32_t copy_last = 0, copy_par = 0;
        // The record ring, allocated here and released in tile order: a
        // record takes [pos, pos + size + 16) of a sequence of positions that
        // maps onto the ring modulo its size (the 16 bytes of slack serve the
        // decoders' 8-byte run reads); it does not wrap around the ring's end
        // but skips the bytes left there.  `freed` is the end of the last
        // released record, `rel` the next tile to be released.
        const uint32_t A = L.ring_bytes;
        unsigned long long a_pos = 0, freed = 0;
        uint32_t a_off = 0, rel = 0;
        bool stop = false;
        // wait until the decoders are done with tile `rel`, and release it
        auto release_one = [&]() {
            const int s2 = (int)(rel % kDSlots);
            if (!mbar_wait_bounded(&consumed[s2], (rel / kDSlots) & 1u, 8 * lc.copy_ns)) {
                stop = true;
                return;
            }
            freed = st_end[s2];
            ++rel;
        };
        // the next tile (its field, local index and index entries), loaded one
        // tile ahead so that its entries arrive while this iteration waits
        uint32_t nf = 0, ntile = 0;
        uint64_t n0 = 0, n1 = 0;
        bool nmore = false;
        // the CTA's i-th tile: a ticket (batches), or its share of the static split
        auto take = [&](uint32_t i) -> uint64_t {
            if constexpr (BATCH) return (uint64_t)atomicAdd(lc.ticket, 1u);
            else return (uint64_t)blockIdx.x + (uint64_t)i * gridDim.x;
        };
        auto load_next = [&](uint64_t t) {
            nmore = t < lc.total_tiles;
            if (!nmore) return;
            nf = dfield_of<BATCH>(lc, t);
            const DField *F = dfield_ptr<BATCH>(one, lc, nf);
            ntile = (uint32_t)(t - F->tile0 + F->tile_lo);
            const uint64_t *idx = reinterpret_cast<const uint64_t *>(F->in + F->g.off_index);
            n0 = idx[ntile];
            n1 = idx[ntile + 1];
        };
        load_next(take(0));
        for (uint32_t it = 0;; ++it) {
            const bool more = nmore;
            const uint32_t f = nf, tile = ntile;
            const DField *F = dfield_ptr<BATCH>(one, lc, f);
            const Geometry &g = F->g;
            const int st = (int)(it % kDSlots);
            const uint32_t k = it / kDSlots;
            const uint64_t r0 = n0, r1 = n1;
            if (more) load_next(take(it + 1));
            if constexpr (!BATCH)
                if (!more) break;  // the static split: the other warps count tiles themselves
            // the slot's previous tile (it - kDSlots) must be released
            while (!stop && rel + kDSlots <= it) release_one();
            if (stop) {
                flag_status(F->status, 6u);
                break;
            }
            if (!more) {
                // no more tickets: the slot carries the end to the other warps
                st_tile[st] = 0xFFFFFFFFu;
                dmbar_arrive(&head[st]);
                dmbar_arrive(&full[st]);
                copy_last &= ~(1u << st);
                break;
            }
            uint32_t bad = 0;
            if (F->check_header && tile == 0) {
                const uint32_t *h32 = reinterpret_cast<const uint32_t *>(F->in);
                const uint64_t *h64 = reinterpret_cast<const uint64_t *>(F->in);
                if (h32[0] != kMagic || (h32[1] & 0xFFFFu) != (kVersion | (F->dtype << 8)) || h32[2] != b ||
                    h32[3] != G || h64[2] != g.n || h64[7] != F->total_bytes)
                    bad = 1;
            }
            if (r0 > r1 || r1 > F->rec_total || (r0 & 15) || (r1 & 15) || r1 - r0 > rec_max) bad = 1;
            if (tile == g.ntiles - 1 && r1 != F->rec_total) bad = 1;
            const uint32_t size = bad ? 0u : (uint32_t)(r1 - r0);
            st_field[st] = f;
            st_tile[st] = tile;
            st_size[st] = size;
            st_bad[st] = bad;
            if (!bad) {
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
                // the record's place in the ring: fits once nothing is held
                // (the skipped bytes are then free as well) or once it ends
                // within one ring of `freed`
                const uint32_t need = size + 16;
                const unsigned long long prev_end = a_pos;
                if (a_off + need > A) {
                    a_pos += A - a_off;
                    a_off = 0;
                }
                const uint32_t r_off = a_off;
                const unsigned long long r_end = a_pos + need;
                while (!stop && rel < it && freed < prev_end && freed + A < r_end) release_one();
                if (stop) {
                    flag_status(F->status, 6u);
                    break;
                }
                a_pos = r_end;
                a_off += need;
                st_off[st] = r_off;
                st_end[st] = r_end;
                uint8_t *rec = smem + L.ring + r_off;
                uint8_t *slot = smem + L.slots + st * L.slot;
                // the head first (what the indexing warp reads: at most
                // G * (b/4 + 1) bytes, rounded up to 16), then the rest
                const uint32_t hb = size < kHeadBytes ? size : kHeadBytes;
                mbar_arrive_expect_tx(&head[st], hb + mu_bytes + (uint32_t)(sbE - sbA));
                bulk_g2s(slot + L.bits, F->in + sbA, (uint32_t)(sbE - sbA), &head[st]);
                if (hb) bulk_g2s(rec, F->in + g.off_rec + r0, hb, &head[st]);
                bulk_g2s(slot + L.mu, F->in + g.off_mu + k0 * w, mu_bytes, &head[st]);
                mbar_arrive_expect_tx(&full[st], size - hb);
                if (size > hb) bulk_g2s(rec + hb, F->in + g.off_rec + r0 + hb, size - hb, &full[st]);
                copy_last |= 1u << st;
                copy_par = (copy_par & ~(1u << st)) | ((k & 1u) << st);
            } else {
                st_end[st] = a_pos;  // no record: releasing the tile frees nothing more
                dmbar_arrive(&head[st]);
                dmbar_arrive(&full[st]);
                copy_last &= ~(1u << st);
            }
        }
        // do not leave while a copy may still be writing into shared memory
        for (int st = 0; st < kDSlots; ++st)
            if ((copy_last >> st) & 1u) {
                mbar_wait_bounded(&head[st], (copy_par >> st) & 1u, lc.copy_ns);
                mbar_wait_bounded(&full[st], (copy_par >> st) & 1u, lc.copy_ns);
            }
        return;
    }

    if (warp == kDIndexerWarp) {
        // ---- indexing warp: per tile, every block's rank among the tile's
        // non-constant blocks, its reqBits byte and the offset of its mid
        // bytes, and the record's checks; ahead of the decoders.
        // Lane l takes blocks BPL*l .. BPL*l + BPL - 1 (consecutive, inside
        // one 32-bit word of state bits), so a scan over lanes orders them.
        constexpr uint32_t BPL = (G + 31) / 32;
        constexpr uint32_t NSW = (G + 31) / 32;  // 32-bit words of state bits
        static_assert(32 % BPL == 0, "a lane's blocks share one state word");
        for (uint32_t it = 0;; ++it) {
            if constexpr (!BATCH)
                if ((uint64_t)blockIdx.x + (uint64_t)it * gridDim.x >= lc.total_tiles) break;
            const int st = (int)(it % kDSlots);
            const uint32_t k = it / kDSlots;
            const bool waited = mbar_wait_bounded(&head[st], k & 1u, lc.copy_ns);
            if (BATCH && waited && st_tile[st] == 0xFFFFFFFFu) {
                // the end: pass it on to the decoders
                if (lane == 0) dmbar_arrive(&indexed[st]);
                break;
            }
            const DField *Fd = dfield_ptr<BATCH>(one, lc, st_field[st]);
            const Geometry &g = Fd->g;
            const uint32_t tile = st_tile[st];
            const uint32_t size = st_size[st];
            const bool pbad = !waited || st_bad[st] != 0;
            const uint8_t *rec = smem + L.ring + st_off[st];
            const uint8_t *slot = smem + L.slots + st * L.slot;
            uint2 *info = reinterpret_cast<uint2 *>(smem + L.slots + st * L.slot + L.info);
            const uint64_t k0 = (uint64_t)tile * G;
            const uint32_t Gt = pbad ? 0u : (uint32_t)min_u64(G, g.nb - k0);

            // the tile's state bits (bits at or past Gt cleared)
            uint32_t sw[NSW];
            {
                const uint8_t *stb = slot + L.bits + st_boff[st];
                if constexpr (G >= 32) {
                    // the tile's bits start at a multiple of 4 bytes
#pragma unroll
                    for (uint32_t i = 0; i < NSW; ++i) sw[i] = reinterpret_cast<const uint32_t *>(stb)[i];
                } else {
                    sw[0] = stb[0];
                    if (G > 8) sw[0] |= (uint32_t)stb[1] << 8;
                }
#pragma unroll
                for (uint32_t i = 0; i < NSW; ++i) {
                    const uint32_t lo = 32 * i;
                    sw[i] &= Gt >= lo + 32 ? kFull : (Gt <= lo ? 0u : (1u << (Gt - lo)) - 1u);
                }
            }
            const uint32_t j0 = (uint32_t)lane * BPL;
            uint32_t nn_t = 0, rank0 = 0, mybits = 0;
#pragma unroll
            for (uint32_t i = 0; i < NSW; ++i) {
                nn_t += __popc(sw[i]);
                if (j0 >= 32 * i + 32) {
                    rank0 += __popc(sw[i]);
                } else if (j0 >= 32 * i) {
                    const uint32_t sh = j0 - 32 * i;
                    rank0 += __popc(sw[i] & ((1u << sh) - 1u));
                    mybits = (sw[i] >> sh) & ((BPL >= 32 ? 0u : (1u << BPL)) - 1u);
                }
            }
            bool ok = (uint64_t)nn_t * (b / 4 + 1) <= size;
            uint32_t rq_b[BPL], rank_b[BPL], mk_b[BPL];
            uint32_t lane_total = 0;
#pragma unroll
            for (uint32_t i = 0; i < BPL; ++i) {
                const uint32_t j = j0 + i;
                const uint32_t rank = rank0 + __popc(mybits & ((1u << i) - 1u));
                const bool ex = j < Gt;
                const uint32_t len = ex ? (uint32_t)min_u64(b, g.n - (k0 + j) * b) : 0u;
                const bool nc = ex && ((mybits >> i) & 1u) && ok;
                const uint32_t rq = nc ? rec[nn_t * (b / 4) + rank] : 0u;
                const bool raw = nc && rq == 0xFFu;
                const bool coded = nc && !raw;
                if (nc && rq == 0u) ok = false;  // 0 marks a constant block in the table
                if (coded && !(rq >= 1u + F::E && rq <= (uint32_t)W)) ok = false;
                const uint32_t s = (8u - (rq & 7u)) & 7u;
                const uint32_t q = coded ? (rq + s) >> 3 : 2u;
                uint32_t suml = 0;
                if (coded) {
                    // the block's codes, b/16 words (16-byte aligned for b >= 64);
                    // codes past the block's end are 0; none exceeds min(3, q)
                    constexpr uint32_t NW = b / 16;
                    constexpr uint32_t VW = NW % 4 == 0 ? 4 : 2;  // words per load
                    const uint8_t *lb = rec + rank * (b / 4);
                    uint32_t any3 = 0, past = 0;
#pragma unroll 2
                    for (uint32_t v4 = 0; v4 < NW / VW; ++v4) {
                        uint32_t c[VW];
                        if constexpr (VW == 4) {
                            const uint4 u = reinterpret_cast<const uint4 *>(lb)[v4];
                            c[0] = u.x, c[1] = u.y, c[2] = u.z, c[3] = u.w;
                        } else {
                            const uint2 u = reinterpret_cast<const uint2 *>(lb)[v4];
                            c[0] = u.x, c[1] = u.y;
                        }
#pragma unroll
                        for (uint32_t e = 0; e < VW; ++e) {
                            any3 |= c[e] & (c[e] >> 1);
                            suml += __popc(c[e]) + __popc(c[e] & 0xAAAAAAAAu);  // lo + 2 hi
                            if (len < b) {
                                const int nv = (int)len - 16 * (int)(v4 * VW + e);
                                const uint32_t vm = nv >= 16 ? kFull : (nv <= 0 ? 0u : (kFull >> (2 * (16 - nv))));
                                past |= c[e] & ~vm;
                            }
                        }
                    }
                    if (past || (q == 2u && (any3 & 0x55555555u))) ok = false;
                }
                const uint32_t mk = coded ? len * q - suml : (raw ? len * w : 0u);
                rq_b[i] = rq;
                rank_b[i] = rank;
                mk_b[i] = mk;
                lane_total += mk;
            }
            uint32_t total;
            const uint32_t excl = warp_exclusive_scan(lane_total, &total);
            const uint32_t used = nn_t * (b / 4 + 1) + total;
            ok = __all_sync(kFull, ok) && !pbad && pad16(used) == size;
            if (ok) {
                uint32_t run = nn_t * (b / 4 + 1) + excl;
#pragma unroll
                for (uint32_t i = 0; i < BPL; ++i) {
                    if (j0 + i < G) info[j0 + i] = make_uint2(run, rank_b[i] | (rq_b[i] << 16));
                    run += mk_b[i];
                }
            }
            if (lane == 0) {
                const uint32_t verdict = ok ? 0u : (!waited ? 6u : 3u);
                st_verdict[st] = verdict;
                st_used[st] = used;
                if (verdict) flag_status(Fd->status, verdict);
                dmbar_arrive(&indexed[st]);
            }
            __syncwarp();
            if (!waited) break;
        }
        return;
    }

    // ---- decoders (warps 0..7) ---------------------------------------------
    uint8_t *wbuf = smem + L.wbuf + warp * L.wbuf_bytes;
    const uint32_t lane_row0 = (uint32_t)(lane * RPL);  // inside the warp's rows
    for (uint32_t it = 0;; ++it) {
        if constexpr (!BATCH)
            if ((uint64_t)blockIdx.x + (uint64_t)it * gridDim.x >= lc.total_tiles) break;
        const int st = (int)(it % kDSlots);
        const uint32_t k = it / kDSlots;
        // the tile's bytes and its block table; a wait that runs out stops
        // this warp
        if (!mbar_wait_bounded(&head[st], k & 1u, lc.copy_ns) || !mbar_wait_bounded(&full[st], k & 1u, lc.copy_ns) ||
            !mbar_wait_bounded(&indexed[st], k & 1u, 2 * lc.copy_ns)) {
            if (lane == 0) flag_status(dfield_ptr<BATCH>(one, lc, st_field[st])->status, 6u);
            break;
        }
        if constexpr (BATCH)
            if (st_tile[st] == 0xFFFFFFFFu) break;  // no more tickets
        const DField *Fd = dfield_ptr<BATCH>(one, lc, st_field[st]);
        const Geometry &g = Fd->g;
        const uint32_t tile = st_tile[st];
        const bool bad = st_verdict[st] != 0;
        const uint8_t *rec = smem + L.ring + st_off[st];
        const uint8_t *slot = smem + L.slots + st * L.slot;
        const uint64_t k0 = (uint64_t)tile * G;
        const uint32_t Gt = (uint32_t)min_u64(G, g.nb - k0);

        // Tiles wholly inside the stream's field and the decoded range, with
        // every output row stored by the tensor copy, run a copy of the work
        // below compiled for that case: no checks of the ends per block, row
        // or group of values
        const bool full_tile = st_verdict[st] == 0 && Fd->use_tma && (k0 + G) * b <= g.n && k0 >= Fd->blk_lo &&
                               k0 + G <= Fd->blk_hi;
        auto tile_body = [&](auto full_c) {
            constexpr bool FT = decltype(full_c)::value;
            const int sub = lane % LPB;
            const uint32_t blk = (uint32_t)(warp * BPW + lane / LPB);
            const bool exists = FT || (blk < Gt && !bad);
            const uint64_t kg = k0 + blk;
            const int len = FT ? (int)b : (exists ? (int)min_u64(b, g.n - kg * b) : 0);
            int nvalid = VPL;
            if constexpr (!FT) {
                nvalid = len - sub * VPL;
                nvalid = nvalid < 0 ? 0 : (nvalid > VPL ? VPL : nvalid);
            }
            const bool full_lane = FT || nvalid == VPL;
            const uint32_t segmask = (LPB == 32 ? kFull : ((1u << LPB) - 1u)) << (lane & ~(LPB - 1));
            U x[VPL];
            if (FT || !bad) {
                // ---- the block's entry: mid-byte offset, rank, reqBits ----------
                const uint2 bi = exists ? reinterpret_cast<const uint2 *>(slot + L.info)[blk] : make_uint2(0, 0);
                const uint32_t mbase = bi.x, rank = bi.y & 0xFFFFu, rq = bi.y >> 16;
                const bool raw = rq == 0xFFu;
                const bool coded = rq != 0u && !raw;
                const int s = (8 - (int)(rq & 7u)) & 7;
                const int q = coded ? ((int)rq + s) >> 3 : 2;
                const int lmax = q < 3 ? q : 3;
                uint32_t codes[NCODE];
#pragma unroll
                for (int i = 0; i < NCODE; ++i) codes[i] = 0;
                if (coded) {
                    const uint8_t *lead = rec + rank * (b / 4) + sub * (VPL / 4);
                    if constexpr (NCODE == 4) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(lead);
                        codes[0] = v.x;
                        codes[1] = v.y;
                        codes[2] = v.z;
                        codes[3] = v.w;
                    } else if constexpr (NCODE == 2) {
                        const uint2 v = *reinterpret_cast<const uint2 *>(lead);
                        codes[0] = v.x;
                        codes[1] = v.y;
                    } else {
                        codes[0] = *reinterpret_cast<const uint32_t *>(lead);
                    }
                }
                const U mu_bits = exists ? reinterpret_cast<const U *>(slot + L.mu)[blk] : U(0);

                // ---- decode --------------------------------------------------
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

                // Does every plane-2 run of the warp hold byte 2 of all its
                // lane's values (no code 3, every value valid)?  Then each
                // group's word of plane 2 is one funnel shift of two
                // consecutive words of the run (one new load per group), with
                // no permute and no carry.  Decided for the whole warp.
                bool dense2;
                {
                    bool no3 = true;
#pragma unroll
                    for (int i = 0; i < NCODE; ++i) no3 = no3 && (codes[i] & (codes[i] >> 1) & 0x55555555u) == 0u;
                    dense2 = __all_sync(kFull, !(coded && q >= 3) || (full_lane && no3));
                }
                if (coded) {
                    const T mu = F::from(mu_bits);
                    // the dense run: 32-bit words from pos2's word on, read with
                    // the byte shift of pos2 (the record's slack covers the last)
                    const uint32_t *rw = reinterpret_cast<const uint32_t *>(rec);
                    const uint32_t w2 = pos2 >> 2, a2 = (pos2 & 3u) * 8u;
                    uint32_t cur2 = (dense2 && q >= 3) ? rw[w2] : 0u;
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
                        // plane words: byte k = byte j of value 4gq + k; a leading
                        // byte takes the nearest earlier owner's, or the carry
                        uint32_t P[W / 8];
#pragma unroll
                        for (int j = 0; j < W / 8; ++j) P[j] = 0;
                        {
                            const uint32_t e0 = lut[code8];
                            P[0] = dprmt(load_run(rec, pos0), carry[0], e0);
                            pos0 += e0 >> 16;
                            carry[0] = P[0] >> 24;
                            const uint32_t e1 = lut[256 + code8];
                            P[1] = dprmt(load_run(rec, pos1), carry[1], e1);
                            pos1 += e1 >> 16;
                            carry[1] = P[1] >> 24;
                            if (q >= 3) {
                                if (dense2) {
                                    const uint32_t nxt = rw[w2 + gq + 1];
                                    P[2] = __funnelshift_r(cur2, nxt, a2);
                                    cur2 = nxt;
                                } else {
                                    const uint32_t e2 = lut[512 + code8];
                                    P[2] = dprmt(load_run(rec, pos2), carry[2], e2);
                                    pos2 += e2 >> 16;
                                    carry[2] = P[2] >> 24;
                                }
                            }
                            if (q >= 4) {
                                // dense planes: every valid value owns its byte
                                const uint32_t sel = full_lane ? 0x3210u : lut[512 + dense8];
#pragma unroll
                                for (int j = 3; j < W / 8; ++j)
                                    if (j < q)
                                        P[j] = dprmt(load_run(rec, dense0 + (uint32_t)(j - 3) * len + 4 * gq), 0, sel);
                            }
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
                // strictness: the record's pad bytes (fewer than 16) must be zero
                if (warp == 0) {
                    const uint32_t used = st_used[st];
                    if (used + lane < st_size[st] && rec[used + lane]) flag_status(Fd->status, 3u);
                }
            }
            // this warp no longer reads the tile's record or slot
            __syncwarp();
            if (lane == 0) dmbar_arrive(&consumed[st]);
            if (!FT && bad) return;

            // ---- output: full rows through the warp's buffer and a tensor store,
            // the ragged last row with plain stores ------------------------------
            // rows of the output count from the range's first row; a warp whose
            // rows all lie at or after it stores through the tensor map (rows past
            // the end are clipped), one that straddles the start stores plainly
            const uint64_t wrow0 = (uint64_t)tile * TILE_ROWS + (uint64_t)warp * 32 * RPL;  // warp's first row
            const bool tma_rows = FT || (Fd->use_tma && wrow0 >= Fd->row_lo && wrow0 - Fd->row_lo < Fd->rows_full);
            const bool wanted = FT || (kg >= Fd->blk_lo && kg < Fd->blk_hi);
            if (tma_rows) {
                // the buffer is free once the previous tile's store has read it
                if (lane == 0) bulk_wait_read_all();
                __syncwarp();
            }
            if (exists && wanted && nvalid > 0) {
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) {
                    constexpr int VPR = 128 / w;  // values per row
                    const int nv = nvalid - rr * VPR;
                    if (nv <= 0) continue;
                    const uint32_t rowi = lane_row0 + rr;
                    if (FT || (tma_rows && wrow0 + rowi - Fd->row_lo < Fd->rows_full)) {
                        uint8_t *row = wbuf + (rowi << 7);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            uint4 v;
                            U *u = reinterpret_cast<U *>(&v);
#pragma unroll
                            for (int kk = 0; kk < 16 / w; ++kk) u[kk] = x[rr * VPR + c * (16 / w) + kk];
                            *reinterpret_cast<uint4 *>(row + ((c ^ (rowi & 7u)) << 4)) = v;
                        }
                    } else {
                        U *dst = reinterpret_cast<U *>(Fd->out) + (kg - Fd->blk_lo) * b + sub * VPL + rr * VPR;
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
            if (tma_rows) {
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    // one store per box of the warp's rows (a box starting past
                    // the range's last row is not issued; rows past it inside a
                    // box are clipped)
#pragma unroll
                    for (uint32_t bx = 0; bx < WARP_BOXES; ++bx) {
                        const uint64_t r0 = wrow0 - Fd->row_lo + bx * BOX_ROWS;
                        if (bx > 0 && !FT && r0 >= Fd->rows_full) break;
                        asm volatile(
                            "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                                reinterpret_cast<uint64_t>(&Fd->tmap)),
                            "r"(0), "r"((int)r0), "r"(smem_addr(wbuf + bx * BOX_ROWS * 128u))
                            : "memory");
                    }
                    bulk_commit();
                }
            }
        };
        if (full_tile) tile_body(std::true_type{});
        else tile_body(std::false_type{});
    }
    // stores must finish reading shared memory (and land) before the CTA leaves
    if (lane == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------

namespace {

template <typename T, int LPB, int VPL, int NDW>
cudaError_t launch_t(const DField &one, const DecompressLaunch &lc, int ctas_per_sm, bool pdl, cudaStream_t stream) {
    constexpr uint32_t b = (uint32_t)(LPB * VPL), w = (uint32_t)Fmt<T>::w;
    const DSmem L = decompress_smem(tile_blocks(b, w), b, w, NDW);
    if (L.ring_bytes < record_max_bytes(tile_blocks(b, w), b, w) + 16) return cudaErrorInvalidValue;
    auto kern =
        lc.fields ? decompress_kernel<T, LPB, VPL, NDW, true> : decompress_kernel<T, LPB, VPL, NDW, false>;
    // per device and kernel: the shared-memory attribute and the occupancy,
    // set up on first use (a launch then only reads them)
    int per_sm = 0, sms = 0;
    cudaError_t err =
        launch_setup(reinterpret_cast<const void *>(kern), L.total, decompress_threads(NDW), &per_sm, &sms);
    if (err != cudaSuccess) return err;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    const uint64_t grid = min_u64(lc.total_tiles, (uint64_t)sms * per_sm);
    return launch_kernel(kern, (unsigned)grid, decompress_threads(NDW), L.total, pdl, stream, one, lc);
}

// The kernel instance for (dtype, block, decoding warps); the same pairs as
// the compressor's.
cudaError_t ddispatch(int dtype, uint32_t block, int nw, const DField &one, const DecompressLaunch &lc,
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

uint64_t copy_limit_ns() { return 1000ull * wait_limit_from_env("SZX_COPY_US", 1000000u); }

}  // namespace

void fill_decompress_field(DField *f, const void *in, uint64_t total_bytes, uint64_t n, int dtype, uint32_t block,
                           void *out, uint32_t *d_status, bool check_header, uint64_t tile0, uint64_t blk_lo,
                           uint64_t blk_hi) {
    DField &a = *f;
    std::memset(&a, 0, sizeof(a));
    const uint32_t w = dtype == 0 ? 4 : 8;
    a.in = static_cast<const uint8_t *>(in);
    a.out = static_cast<uint8_t *>(out);
    a.status = d_status;
    a.g = make_geometry(n, block, w);
    a.rec_total = total_bytes - a.g.off_rec;
    a.total_bytes = total_bytes;
    if (blk_hi > a.g.nb) blk_hi = a.g.nb;
    a.blk_lo = blk_lo;
    a.blk_hi = blk_hi;
    a.tile_lo = blk_lo / a.g.G;
    a.row_lo = blk_lo * block * w / 128;  // b * w is a multiple of 128
    const uint64_t range_vals = min_u64(n, blk_hi * block) - blk_lo * block;
    a.rows_full = range_vals * w / 128;
    a.tile0 = tile0;
    a.dtype = (uint32_t)dtype;
    a.check_header = check_header ? 1u : 0u;
    // boxes of an eighth of a tile's rows: one per warp of eight (their 32
    // lanes' rows), two per warp of four
    const uint32_t box_rows = (dtype == 1 && block == 1024) ? 64u : 32u;
    a.use_tma = encode_row_map(&a.tmap, out, a.rows_full, box_rows) ? 1u : 0u;
}

uint64_t decompress_field_tiles(const DField *f) {
    return f->blk_hi > f->blk_lo ? (f->blk_hi - 1) / f->g.G - f->tile_lo + 1 : 0;
}

cudaError_t launch_decompress(const void *in, uint64_t in_bytes, uint64_t total_bytes, uint64_t n, int dtype,
                              uint32_t block, void *out, uint32_t *d_status, bool check_header,
                              cudaStream_t stream, uint64_t blk_lo, uint64_t blk_hi, Clear clear) {
    (void)in_bytes;
    DField one;
    fill_decompress_field(&one, in, total_bytes, n, dtype, block, out, d_status, check_header, 0, blk_lo, blk_hi);
    DecompressLaunch lc;
    lc.fields = nullptr;
    lc.nfields = 1;
    lc.total_tiles = decompress_field_tiles(&one);
    // the status starts at zero; with the clear kernel, the decoder starts
    // behind it
    if (clear == Clear::automatic) clear = lc.total_tiles >= kClearKernelMinTiles ? Clear::kernel : Clear::memset;
    if (d_status) {
        const cudaError_t err = clear == Clear::memset ? cudaMemsetAsync(d_status, 0, sizeof(uint32_t), stream)
                                                       : launch_clear_words(d_status, 1, stream);
        if (err != cudaSuccess) return err;
    }
    if (!lc.total_tiles) return cudaSuccess;
    lc.copy_ns = copy_limit_ns();
    lc.ticket = nullptr;  // no device workspace here: the static split
    return ddispatch(dtype, block, 8, one, lc, 0, d_status != nullptr && clear == Clear::kernel, stream);
}

cudaError_t launch_decompress_batch(const void *d_fields, uint32_t nfields, uint64_t total_tiles, uint32_t *d_ticket,
                                    int dtype, uint32_t block, int ctas_per_sm, int nw, bool pdl,
                                    cudaStream_t stream) {
    DField one;
    std::memset(&one, 0, sizeof(one));
    DecompressLaunch lc;
    lc.fields = static_cast<const DField *>(d_fields);
    lc.nfields = nfields;
    lc.total_tiles = total_tiles;
    lc.copy_ns = copy_limit_ns();
    lc.ticket = d_ticket;
    return ddispatch(dtype, block, nw, one, lc, ctas_per_sm, pdl, stream);
}

}  // namespace szx
