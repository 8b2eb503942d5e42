// batch.cu -- batched compression and decompression (many fields, few launches).
//
// A plan groups the fields by (dtype, block): each group is one persistent
// launch of the same kernels as the single-field calls, over the global list
// of all its fields' tiles, handed out by one ticket counter per group, with
// the per-field descriptors in a table in device memory.  The caller's
// workspace holds, in order:
//   descriptor tables (one CField or DField per field, 64-byte aligned),
//   per-group counters (ticket, done, error: 16 bytes each; decompression
//   uses the ticket only),
//   per-field compression workspaces (counters + look-back words, 256-byte
//   aligned; compression only).
// Running a plan is one clear kernel (counters, workspaces and, for
// decompression, every stream's status word) plus one kernel launch per group,
// each the programmatic dependent of the kernel before it, so it can be
// captured in a CUDA graph once the tables are uploaded.  The autotuner times
// each group alone on the plan's own
// data in every shape the kernels have -- consumer warps per CTA (8, or 4 with
// twice the values per lane and blocks per warp) times CTAs per SM (2 or 1) --
// and keeps the fastest; the stream is the same in every shape.  For a group
// of fields given block 0 it also tries the block lengths 64, 128 and 256
// (which do change the stream), and among those within 2% of the fastest time
// keeps the one that writes the fewest bytes.
#include "szx.h"
#include "szx_device.cuh"
#include "szx_host.h"
#include "szx_launch.h"

#include <algorithm>
#include <iterator>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using namespace szx;

namespace {

// A run's state cleared in one kernel: n words at `words` (the plan's counters
// and, for compression, the fields' workspaces) and, for decompression, the
// status word of each of the nfields descriptors at `fields` (device memory).
// The first group's launch follows it as its programmatic dependent.
__global__ void clear_run_kernel(uint32_t *words, uint64_t n, const DField *fields, uint32_t nfields) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = i0; i < n; i += stride) words[i] = 0u;
    if (fields)
        for (uint64_t i = i0; i < nfields; i += stride) {
            uint32_t *st = fields[i].status;
            if (st) *st = 0u;
        }
}

struct Group {
    int dtype;
    uint32_t block;
    uint32_t first, count;  // slice of the (grouped) table
    uint64_t tiles;
    int ctas_per_sm;  // 0: as many as fit
    int nw;           // consumer (decoding) warps per CTA: 8 or 4
    bool auto_block;  // its fields asked for block 0: the tuner picks b
    float tuned_ms;   // the tuner's best time for the group (0: not tuned)
};

// Block lengths the tuner tries for block-0 fields (and the one used until it
// runs).  For each of them a tile holds the same number of values (32 KiB),
// so a field's tile count and workspace do not depend on the choice.
constexpr uint32_t kAutoBlocks[3] = {64, 128, 256};
constexpr uint32_t kAutoDefault = 128;

}  // namespace

struct szx_batch_plan {
    bool compress;
    std::vector<szx_field> fields;          // compression: the caller's fields
    std::vector<szx_stream_field> streams;  // decompression: the caller's streams
    std::vector<uint32_t> order;            // table slot -> caller's index
    std::vector<Group> groups;
    std::vector<uint64_t> ws_off;  // compression: per table slot, its workspace offset
    uint64_t table_bytes = 0, counters_off = 0, zero_off = 0, total_bytes = 0;
    void *uploaded_ws = nullptr;  // the workspace the tables were written to
    uint64_t *uploaded_results = nullptr;  // and the results array given then
};

namespace {

szx_status make_groups(szx_batch_plan *p, const std::vector<std::pair<int, uint32_t>> &keys,
                       const std::vector<uint64_t> &tiles) {
    const uint32_t n = (uint32_t)keys.size();
    p->order.resize(n);
    for (uint32_t i = 0; i < n; ++i) p->order[i] = i;
    std::stable_sort(p->order.begin(), p->order.end(), [&](uint32_t a, uint32_t b) { return keys[a] < keys[b]; });
    for (uint32_t s = 0; s < n;) {
        Group g;
        g.dtype = keys[p->order[s]].first;
        g.block = keys[p->order[s]].second;
        g.first = s;
        g.tiles = 0;
        g.ctas_per_sm = 0;
        g.nw = 8;
        g.tuned_ms = 0.0f;
        while (s < n && keys[p->order[s]] == std::make_pair(g.dtype, g.block)) g.tiles += tiles[p->order[s++]];
        g.count = s - g.first;
        g.auto_block = g.block == 0;
        if (g.auto_block) g.block = kAutoDefault;
        if (g.tiles >= (1ull << 32)) return SZX_ERR_INVALID;  // tickets are 32-bit
        p->groups.push_back(g);
    }
    return SZX_OK;
}

}  // namespace

extern "C" {

szx_status szx_batch_compress_plan(const szx_field *fields, int count, szx_batch_plan **plan) {
    if (!plan) return SZX_ERR_INVALID;
    *plan = nullptr;
    if (!fields || count <= 0) return SZX_ERR_INVALID;
    szx_batch_plan *p = new (std::nothrow) szx_batch_plan;
    if (!p) return SZX_ERR_NOMEM;
    p->compress = true;
    std::vector<std::pair<int, uint32_t>> keys;
    std::vector<uint64_t> tiles;
    for (int i = 0; i < count; ++i) {
        const szx_field &f = fields[i];
        // block 0: the largest stream over the tuner's candidates
        size_t smax = 0;
        if (f.block == 0) {
            for (uint32_t b : kAutoBlocks) {
                const size_t m = szx_stream_max_bytes(f.n, f.dtype, b);
                if (!m) {  // an invalid field
                    smax = 0;
                    break;
                }
                smax = m > smax ? m : smax;
            }
        } else {
            smax = szx_stream_max_bytes(f.n, f.dtype, f.block);
        }
        if (!f.d_in || !f.d_out || !smax || !aligned16(f.d_in) || !aligned16(f.d_out) || !(f.eb > 0.0) ||
            !std::isfinite(f.eb)) {
            delete p;
            return SZX_ERR_INVALID;
        }
        if (f.out_capacity < smax) {
            delete p;
            return SZX_ERR_TOO_SMALL;
        }
        p->fields.push_back(f);
        keys.emplace_back((int)f.dtype, f.block);
        tiles.push_back(make_geometry(f.n, f.block ? f.block : kAutoDefault, f.dtype == SZX_F32 ? 4 : 8).ntiles);
    }
    szx_status st = make_groups(p, keys, tiles);
    if (st != SZX_OK) {
        delete p;
        return st;
    }
    p->table_bytes = align_up((uint64_t)count * sizeof(CField), 256);
    p->counters_off = p->table_bytes;
    p->zero_off = p->counters_off;
    uint64_t o = p->counters_off + align_up(16 * p->groups.size(), 256);
    p->ws_off.resize(count);
    for (int s = 0; s < count; ++s) {
        p->ws_off[s] = o;
        o += align_up(workspace_bytes(tiles[p->order[s]]), 256);
    }
    p->total_bytes = o;
    *plan = p;
    return SZX_OK;
}

szx_status szx_batch_decompress_plan(const szx_stream_field *streams, int count, szx_batch_plan **plan) {
    if (!plan) return SZX_ERR_INVALID;
    *plan = nullptr;
    if (!streams || count <= 0) return SZX_ERR_INVALID;
    szx_batch_plan *p = new (std::nothrow) szx_batch_plan;
    if (!p) return SZX_ERR_NOMEM;
    p->compress = false;
    std::vector<std::pair<int, uint32_t>> keys;
    std::vector<uint64_t> tiles;
    for (int i = 0; i < count; ++i) {
        const szx_stream_field &s = streams[i];
        const szx_header &h = s.header;
        const bool dt_ok = h.dtype == SZX_F32 || h.dtype == SZX_F64;
        if (!s.d_in || !s.d_out || !aligned16(s.d_in) || !aligned16(s.d_out) || !dt_ok || !block_ok(h.block) ||
            h.n == 0 || h.n > (1ull << 40) || h.tile_blocks != tile_blocks(h.block, h.dtype == SZX_F32 ? 4 : 8)) {
            delete p;
            return SZX_ERR_INVALID;
        }
        const Geometry g = make_geometry(h.n, h.block, h.dtype == SZX_F32 ? 4 : 8);
        if (h.total_bytes > s.in_bytes || h.total_bytes < g.off_rec) {
            delete p;
            return SZX_ERR_CORRUPT;
        }
        if (s.out_capacity < h.n * (h.dtype == SZX_F32 ? 4 : 8)) {
            delete p;
            return SZX_ERR_TOO_SMALL;
        }
        p->streams.push_back(s);
        keys.emplace_back((int)h.dtype, h.block);
        tiles.push_back(g.ntiles);
    }
    szx_status st = make_groups(p, keys, tiles);
    if (st != SZX_OK) {
        delete p;
        return st;
    }
    p->table_bytes = align_up((uint64_t)count * sizeof(DField), 256);
    // per group, a tile ticket (16 bytes, as for compression), zeroed per run
    p->counters_off = p->zero_off = p->table_bytes;
    p->total_bytes = p->counters_off + align_up(16 * p->groups.size(), 256);
    *plan = p;
    return SZX_OK;
}

size_t szx_batch_workspace_bytes(const szx_batch_plan *plan) { return plan ? (size_t)plan->total_bytes : 0; }

szx_status szx_batch_upload(szx_batch_plan *p, void *d_ws, size_t ws_bytes, uint64_t *d_results,
                            szx_stream_t stream) {
    if (!p || !d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return SZX_ERR_INVALID;
    if (ws_bytes < p->total_bytes) return SZX_ERR_TOO_SMALL;
    uint8_t *base = static_cast<uint8_t *>(d_ws);
    const uint32_t n = (uint32_t)p->order.size();
    std::vector<uint8_t> host(p->table_bytes, 0);
    for (const Group &g : p->groups) {
        uint64_t tile0 = 0;
        for (uint32_t s = g.first; s < g.first + g.count; ++s) {
            const uint32_t i = p->order[s];
            if (p->compress) {
                const szx_field &f = p->fields[i];
                CField *c = reinterpret_cast<CField *>(host.data()) + s;
                fill_compress_field(c, f.d_in, f.n, (int)f.dtype, bound_bits(f.eb, f.dtype), g.block, f.d_out,
                                    base + p->ws_off[s], d_results ? d_results + 2 * i : nullptr, tile0);
                tile0 += c->g.ntiles;
            } else {
                const szx_stream_field &sf = p->streams[i];
                DField *d = reinterpret_cast<DField *>(host.data()) + s;
                fill_decompress_field(d, sf.d_in, sf.header.total_bytes, sf.header.n, (int)sf.header.dtype,
                                      sf.header.block, sf.d_out, sf.d_status, true, tile0);
                tile0 += decompress_field_tiles(d);
            }
        }
    }
    (void)n;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(base, host.data(), p->table_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SZX_ERR_CUDA;
    // the staging buffer goes out of scope: make sure the copy has read it
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZX_ERR_CUDA;
    p->uploaded_ws = d_ws;
    p->uploaded_results = d_results;
    return SZX_OK;
}

szx_status szx_batch_run(const szx_batch_plan *p, void *d_ws, szx_stream_t stream) {
    if (!p || !d_ws) return SZX_ERR_INVALID;
    if (d_ws != p->uploaded_ws) return SZX_ERR_INVALID;  // the tables point into that workspace
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *base = static_cast<uint8_t *>(d_ws);
    // counters (and, for compression, the fields' workspaces) start at zero,
    // and so does every stream's status word (SZX_OK); the region is a whole
    // number of 256-byte units
    {
        const uint64_t nwords = (p->total_bytes - p->zero_off) / 4;
        const uint32_t nst = p->compress ? 0u : (uint32_t)p->streams.size();
        const uint64_t items = nwords > nst ? nwords : nst;
        const uint64_t ctas = std::min<uint64_t>((items + 255) / 256, 4 * 148);
        clear_run_kernel<<<(unsigned)(ctas ? ctas : 1), 256, 0, s>>>(
            reinterpret_cast<uint32_t *>(base + p->zero_off), nwords,
            p->compress ? nullptr : reinterpret_cast<const DField *>(base), nst);
        if (cudaGetLastError() != cudaSuccess) return SZX_ERR_CUDA;
    }
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        const Group &g = p->groups[gi];
        cudaError_t e;
        if (p->compress) {
            const CField *tbl = reinterpret_cast<const CField *>(base) + g.first;
            uint32_t *ctr = reinterpret_cast<uint32_t *>(base + p->counters_off + 16 * gi);
            e = launch_compress_batch(tbl, g.count, g.tiles, ctr, g.dtype, g.block, g.ctas_per_sm, g.nw, true, s);
        } else {
            const DField *tbl = reinterpret_cast<const DField *>(base) + g.first;
            uint32_t *ticket = reinterpret_cast<uint32_t *>(base + p->counters_off + 16 * gi);
            e = launch_decompress_batch(tbl, g.count, g.tiles, ticket, g.dtype, g.block, g.ctas_per_sm, g.nw, true,
                                        s);
        }
        if (e != cudaSuccess) return SZX_ERR_CUDA;
    }
    return SZX_OK;
}

szx_status szx_batch_autotune(szx_batch_plan *p, void *d_ws, szx_stream_t stream) {
    if (!p || !d_ws || d_ws != p->uploaded_ws) return SZX_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SZX_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SZX_ERR_CUDA;
    }
    szx_status st = SZX_OK;
    // the fastest of three runs of group gi alone in its current shape (ms)
    auto time_group = [&](size_t gi, float *ms) {
        szx_batch_plan one = *p;
        one.groups.assign(1, p->groups[gi]);
        float t_min = 0.0f;
        for (int r = 0; r < 3; ++r) {
            if (cudaEventRecord(e0, s) != cudaSuccess) return SZX_ERR_CUDA;
            szx_status rs = szx_batch_run(&one, d_ws, stream);
            if (rs != SZX_OK) return rs;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return SZX_ERR_CUDA;
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (r == 0 || t < t_min) t_min = t;
        }
        *ms = t_min;
        return SZX_OK;
    };
    // the group's stream bytes after a run (each stream's header holds its size)
    auto group_bytes = [&](size_t gi, uint64_t *bytes) {
        const Group &g = p->groups[gi];
        uint64_t sum = 0;
        for (uint32_t t = g.first; t < g.first + g.count; ++t) {
            uint64_t total = 0;
            const uint8_t *h = static_cast<const uint8_t *>(p->fields[p->order[t]].d_out);
            if (cudaMemcpyAsync(&total, h + 56, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return SZX_ERR_CUDA;
            sum += total;
        }
        *bytes = sum;
        return SZX_OK;
    };
    for (size_t gi = 0; gi < p->groups.size() && st == SZX_OK; ++gi) {
        Group &g = p->groups[gi];
        std::vector<uint32_t> blocks;
        if (p->compress && g.auto_block) blocks.assign(std::begin(kAutoBlocks), std::end(kAutoBlocks));
        else blocks.assign(1, g.block);
        struct Choice {
            uint32_t block;
            int nw, ctas;
            float ms;
            uint64_t bytes;
        };
        std::vector<Choice> best;  // per block length, its fastest shape
        for (uint32_t b : blocks) {
            if (b != g.block) {
                g.block = b;  // the tables name the block length: write them again
                st = szx_batch_upload(p, d_ws, p->total_bytes, p->uploaded_results, stream);
                if (st != SZX_OK) break;
            }
            Choice c{b, 8, 0, 0.0f, 0};
            for (int nw : {8, 4}) {
                if (!kernel_shape_ok(g.dtype, b, nw)) continue;
                for (int ctas : {2, 1}) {
                    g.nw = nw;
                    g.ctas_per_sm = ctas;
                    float ms = 0.0f;
                    st = time_group(gi, &ms);
                    if (st != SZX_OK) break;
                    if (c.ms == 0.0f || ms < c.ms) {
                        c.nw = nw;
                        c.ctas = ctas;
                        c.ms = ms;
                    }
                }
                if (st != SZX_OK) break;
            }
            if (st != SZX_OK) break;
            if (p->compress && blocks.size() > 1) st = group_bytes(gi, &c.bytes);
            if (st != SZX_OK) break;
            best.push_back(c);
        }
        if (st != SZX_OK) break;
        // the fastest shape; among block lengths within 2% of the fastest
        // time, the one that writes the fewest bytes (the best ratio)
        float t_best = best[0].ms;
        for (const Choice &c : best) t_best = c.ms < t_best ? c.ms : t_best;
        const Choice *pick = nullptr;
        for (const Choice &c : best) {
            if (c.ms > 1.02f * t_best) continue;
            if (!pick || c.bytes < pick->bytes || (c.bytes == pick->bytes && c.ms < pick->ms)) pick = &c;
        }
        g.nw = pick->nw;
        g.ctas_per_sm = pick->ctas;
        g.tuned_ms = pick->ms;
        if (pick->block != g.block) {
            g.block = pick->block;
            st = szx_batch_upload(p, d_ws, p->total_bytes, p->uploaded_results, stream);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

szx_status szx_batch_group_info(const szx_batch_plan *p, int group, szx_batch_group *info) {
    if (!p || !info || group < 0 || group >= (int)p->groups.size()) return SZX_ERR_INVALID;
    const Group &g = p->groups[group];
    const uint32_t w = g.dtype == SZX_F32 ? 4u : 8u;
    const uint32_t G = tile_blocks(g.block, w);
    info->dtype = (szx_dtype)g.dtype;
    info->block = g.block;
    info->auto_block = g.auto_block ? 1 : 0;
    info->fields = g.count;
    info->tiles = g.tiles;
    info->ctas_per_sm = g.ctas_per_sm;
    info->warps_per_cta = g.nw;
    info->threads_per_cta = (uint32_t)g.nw * 32u + 64u;
    info->values_per_lane = G * g.block / (32u * (uint32_t)g.nw);
    info->blocks_per_warp = 32u * info->values_per_lane >= g.block ? 32u * info->values_per_lane / g.block : 0u;
    info->tuned_ms = g.tuned_ms;
    return SZX_OK;
}

szx_status szx_batch_set_group(szx_batch_plan *p, int group, int ctas_per_sm, int warps_per_cta) {
    if (!p || group < 0 || group >= (int)p->groups.size() || ctas_per_sm < 0 || ctas_per_sm > 2) return SZX_ERR_INVALID;
    Group &g = p->groups[group];
    if (!kernel_shape_ok(g.dtype, g.block, warps_per_cta)) return SZX_ERR_INVALID;
    g.ctas_per_sm = ctas_per_sm;
    g.nw = warps_per_cta;
    return SZX_OK;
}

int szx_batch_groups(const szx_batch_plan *p, int *ctas_per_sm, int capacity) {
    if (!p) return 0;
    for (int i = 0; i < capacity && i < (int)p->groups.size(); ++i) ctas_per_sm[i] = p->groups[i].ctas_per_sm;
    return (int)p->groups.size();
}

void szx_batch_destroy(szx_batch_plan *p) { delete p; }

}  // extern "C"
