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
// Running a plan is one cudaMemsetAsync (counters and workspaces) plus one
// kernel launch per group, so it can be captured in a CUDA graph once the
// tables are uploaded.  The autotuner picks, per group, how many CTAs share an
// SM (the kernels fit one or two) by timing both on the plan's own data; the
// streams it writes are the same either way.
#include "szx.h"
#include "szx_device.cuh"
#include "szx_host.h"
#include "szx_launch.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using namespace szx;

namespace {

struct Group {
    int dtype;
    uint32_t block;
    uint32_t first, count;  // slice of the (grouped) table
    uint64_t tiles;
    int ctas_per_sm;  // 0: as many as fit
};

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
        while (s < n && keys[p->order[s]] == std::make_pair(g.dtype, g.block)) g.tiles += tiles[p->order[s++]];
        g.count = s - g.first;
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
        const size_t smax = szx_stream_max_bytes(f.n, f.dtype, f.block);
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
        tiles.push_back(make_geometry(f.n, f.block, f.dtype == SZX_F32 ? 4 : 8).ntiles);
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
                fill_compress_field(c, f.d_in, f.n, (int)f.dtype, bound_bits(f.eb, f.dtype), f.block, f.d_out,
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
    return SZX_OK;
}

szx_status szx_batch_run(const szx_batch_plan *p, void *d_ws, szx_stream_t stream) {
    if (!p || !d_ws) return SZX_ERR_INVALID;
    if (d_ws != p->uploaded_ws) return SZX_ERR_INVALID;  // the tables point into that workspace
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *base = static_cast<uint8_t *>(d_ws);
    // counters (and, for compression, the fields' workspaces) start at zero
    if (cudaMemsetAsync(base + p->zero_off, 0, p->total_bytes - p->zero_off, s) != cudaSuccess) return SZX_ERR_CUDA;
    if (!p->compress) {
        // every stream's status word starts at SZX_OK
        for (const szx_stream_field &sf : p->streams)
            if (sf.d_status && cudaMemsetAsync(sf.d_status, 0, sizeof(uint32_t), s) != cudaSuccess)
                return SZX_ERR_CUDA;
    }
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        const Group &g = p->groups[gi];
        cudaError_t e;
        if (p->compress) {
            const CField *tbl = reinterpret_cast<const CField *>(base) + g.first;
            uint32_t *ctr = reinterpret_cast<uint32_t *>(base + p->counters_off + 16 * gi);
            e = launch_compress_batch(tbl, g.count, g.tiles, ctr, g.dtype, g.block, g.ctas_per_sm, s);
        } else {
            const DField *tbl = reinterpret_cast<const DField *>(base) + g.first;
            uint32_t *ticket = reinterpret_cast<uint32_t *>(base + p->counters_off + 16 * gi);
            e = launch_decompress_batch(tbl, g.count, g.tiles, ticket, g.dtype, g.block, g.ctas_per_sm, s);
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
    for (size_t gi = 0; gi < p->groups.size() && st == SZX_OK; ++gi) {
        float best = 0.0f;
        int best_c = 0;
        for (int c : {2, 1}) {
            // the group alone, c CTAs per SM; the fastest of three runs
            szx_batch_plan one = *p;
            one.groups.assign(1, p->groups[gi]);
            one.groups[0].ctas_per_sm = c;
            float t_min = 0.0f;
            for (int r = 0; r < 3; ++r) {
                if (cudaEventRecord(e0, s) != cudaSuccess) st = SZX_ERR_CUDA;
                if (st == SZX_OK) st = szx_batch_run(&one, d_ws, stream);
                if (st == SZX_OK && cudaEventRecord(e1, s) != cudaSuccess) st = SZX_ERR_CUDA;
                if (st == SZX_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SZX_ERR_CUDA;
                if (st != SZX_OK) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r == 0 || ms < t_min) t_min = ms;
            }
            if (st != SZX_OK) break;
            if (best_c == 0 || t_min < best) {
                best = t_min;
                best_c = c;
            }
        }
        if (st == SZX_OK) p->groups[gi].ctas_per_sm = best_c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

int szx_batch_groups(const szx_batch_plan *p, int *ctas_per_sm, int capacity) {
    if (!p) return 0;
    for (int i = 0; i < capacity && i < (int)p->groups.size(); ++i) ctas_per_sm[i] = p->groups[i].ctas_per_sm;
    return (int)p->groups.size();
}

void szx_batch_destroy(szx_batch_plan *p) { delete p; }

}  // extern "C"
