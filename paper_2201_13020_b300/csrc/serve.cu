// serve.cu -- the serving loop: compress / decompress requests that arrive
// over time, with compressed streams kept resident in a device memory pool.
//
// Continuous batching on one GPU.  A request is admitted as soon as a slot (a
// CUDA stream of the server) and room in the pool are free, oldest first, so
// requests that arrive while others run join them and overlap on the device.
// The loop never synchronises the device:
//   - a compression writes its {stream bytes, status} into pinned, mapped host
//     memory (szx_compress_async's result pointer), read once the slot's event
//     has completed; its pool block is then shrunk to the stream's size (the
//     look-back scratch tail is given back) and the stream stays resident;
//   - a decompression of a resident stream is launched with the header the
//     server already knows from the compression (no device-to-host read); its
//     status word is copied to pinned memory on the same stream before the
//     event.
// The pool itself is the caller's device buffer: the server only keeps the
// bookkeeping of its free ranges (first fit, 256-byte granules, coalescing).
#include "szx.h"
#include "szx_device.cuh"
#include "szx_launch.h"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <numeric>
#include <vector>

using namespace szx;

namespace {

constexpr uint64_t kGranule = 256;
uint64_t granules(uint64_t n) { return (n + kGranule - 1) / kGranule * kGranule; }

}  // namespace

struct szx_server {
    uint8_t *pool = nullptr;
    uint64_t pool_bytes = 0;
    std::map<uint64_t, uint64_t> free;  // offset -> length, disjoint, coalesced
    uint64_t used = 0;
    int slots = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    uint64_t *h_results = nullptr;  // pinned, mapped: 2 per slot
    uint64_t *d_results = nullptr;  // its device address
    uint32_t *d_status = nullptr;   // device: 1 per slot
    uint32_t *h_status = nullptr;   // pinned: 1 per slot

    bool alloc(uint64_t nbytes, uint64_t *off) {
        const uint64_t n = granules(nbytes ? nbytes : 1);
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n, at = it->first + n;
                free.erase(it);
                if (rest) free.emplace(at, rest);
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t nbytes) {
        uint64_t n = granules(nbytes ? nbytes : 1);
        used -= n;
        auto next = free.lower_bound(off);
        if (next != free.end() && off + n == next->first) {
            n += next->second;
            next = free.erase(next);
        }
        if (next != free.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free.emplace(off, n);
    }
    void shrink(uint64_t off, uint64_t old_bytes, uint64_t new_bytes) {
        const uint64_t a = granules(new_bytes ? new_bytes : 1), b = granules(old_bytes ? old_bytes : 1);
        if (b > a) release(off + a, b - a);
    }
};

extern "C" {

szx_status szx_server_create(void *d_pool, size_t pool_bytes, int slots, szx_server **out) {
    if (!out) return SZX_ERR_INVALID;
    *out = nullptr;
    if (!d_pool || (reinterpret_cast<uintptr_t>(d_pool) & (kGranule - 1)) || pool_bytes < kGranule || slots < 1 ||
        slots > 64)
        return SZX_ERR_INVALID;
    szx_server *s = new (std::nothrow) szx_server;
    if (!s) return SZX_ERR_NOMEM;
    s->pool = static_cast<uint8_t *>(d_pool);
    s->pool_bytes = pool_bytes / kGranule * kGranule;
    s->free.emplace(0, s->pool_bytes);
    s->slots = slots;
    bool ok = cudaHostAlloc(&s->h_results, 2 * sizeof(uint64_t) * slots, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->d_results), s->h_results, 0) == cudaSuccess &&
              cudaHostAlloc(&s->h_status, sizeof(uint32_t) * slots, cudaHostAllocDefault) == cudaSuccess &&
              cudaMalloc(&s->d_status, sizeof(uint32_t) * slots) == cudaSuccess;
    for (int i = 0; ok && i < slots; ++i) {
        cudaStream_t st;
        cudaEvent_t ev;
        ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) s->streams.push_back(st);
        ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok) s->events.push_back(ev);
    }
    if (!ok) {
        szx_server_destroy(s);
        return SZX_ERR_CUDA;
    }
    *out = s;
    return SZX_OK;
}

void *szx_server_pool(const szx_server *s) { return s ? s->pool : nullptr; }

size_t szx_server_free_bytes(const szx_server *s) { return s ? (size_t)(s->pool_bytes - s->used) : 0; }

szx_status szx_server_release(szx_server *s, uint64_t offset, uint64_t bytes) {
    if (!s || offset % kGranule || offset + granules(bytes) > s->pool_bytes) return SZX_ERR_INVALID;
    s->release(offset, bytes);
    return SZX_OK;
}

szx_status szx_server_run(szx_server *s, szx_request *reqs, int count, int *max_in_flight) {
    if (!s || (!reqs && count) || count < 0) return SZX_ERR_INVALID;
    using clock = std::chrono::steady_clock;
    const auto t0 = clock::now();
    auto now = [&] { return std::chrono::duration<double>(clock::now() - t0).count(); };

    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return reqs[a].arrival_s < reqs[b].arrival_s; });
    std::vector<char> done(count, 0);
    for (int i = 0; i < count; ++i) {
        reqs[i].status = -1;
        reqs[i].admit_s = reqs[i].done_s = -1.0;
        reqs[i].offset = reqs[i].bytes = 0;
    }
    // a decompression must name an earlier compression that arrives before it
    // (so that first-come-first-served admission reaches the source first)
    for (int i = 0; i < count; ++i) {
        szx_request &r = reqs[i];
        if (r.kind != SZX_REQ_DECOMPRESS) continue;
        const bool ok = r.source >= 0 && r.source < i && reqs[r.source].kind == SZX_REQ_COMPRESS &&
                        reqs[r.source].arrival_s <= r.arrival_s;
        if (!ok) {
            r.status = SZX_ERR_INVALID;
            r.admit_s = r.done_s = 0.0;
            done[i] = 1;
        }
    }
    size_t next = 0;
    std::deque<int> waiting;
    std::vector<int> slot_req(s->slots, -1);
    std::vector<uint64_t> slot_off(s->slots, 0), slot_need(s->slots, 0);
    std::vector<int> idle;
    for (int i = s->slots - 1; i >= 0; --i) idle.push_back(i);
    int running = 0, peak = 0;
    szx_status result = SZX_OK;

    auto finish = [&](int slot, cudaError_t qe) {
        szx_request &r = reqs[slot_req[slot]];
        r.done_s = now();
        if (qe != cudaSuccess) {
            r.status = SZX_ERR_CUDA;
            s->release(slot_off[slot], slot_need[slot]);
        } else if (r.kind == SZX_REQ_COMPRESS) {
            volatile uint64_t *res = s->h_results + 2 * slot;
            r.status = (int)res[1];
            r.bytes = res[0];
            if (r.status == SZX_OK) {
                s->shrink(slot_off[slot], slot_need[slot], r.bytes);
                r.offset = slot_off[slot];
            } else {
                s->release(slot_off[slot], slot_need[slot]);
            }
        } else {
            r.status = (int)(volatile uint32_t &)s->h_status[slot];
            r.bytes = slot_need[slot];
            if (r.keep_output && r.status == SZX_OK) r.offset = slot_off[slot];
            else s->release(slot_off[slot], slot_need[slot]);
        }
        done[slot_req[slot]] = 1;
        slot_req[slot] = -1;
        idle.push_back(slot);
        --running;
    };

    while (next < order.size() || !waiting.empty() || running) {
        const double t = now();
        while (next < order.size() && reqs[order[next]].arrival_s <= t) {
            const int i = order[next++];
            if (!done[i]) waiting.push_back(i);
        }
        for (int slot = 0; slot < s->slots; ++slot) {
            if (slot_req[slot] < 0) continue;
            const cudaError_t qe = cudaEventQuery(s->events[slot]);
            if (qe != cudaErrorNotReady) finish(slot, qe);
        }
        while (!waiting.empty() && !idle.empty()) {
            const int i = waiting.front();
            szx_request &r = reqs[i];
            uint64_t need;
            szx_header h;
            if (r.kind == SZX_REQ_COMPRESS) {
                need = szx_compress_bound(r.n, r.dtype, r.block);
                if (!need) {
                    r.status = SZX_ERR_INVALID;
                    r.admit_s = r.done_s = now();
                    done[i] = 1;
                    waiting.pop_front();
                    continue;
                }
            } else {
                if (r.source < 0 || r.source >= count || reqs[r.source].kind != SZX_REQ_COMPRESS) {
                    r.status = SZX_ERR_INVALID;
                    r.admit_s = r.done_s = now();
                    done[i] = 1;
                    waiting.pop_front();
                    continue;
                }
                const szx_request &src = reqs[r.source];
                if (!done[r.source]) break;  // its stream is not there yet
                if (src.status != SZX_OK) {
                    r.status = src.status;
                    r.admit_s = r.done_s = now();
                    done[i] = 1;
                    waiting.pop_front();
                    continue;
                }
                std::memset(&h, 0, sizeof(h));
                h.block = src.block;
                h.dtype = src.dtype;
                h.n = src.n;
                h.tile_blocks = tile_blocks(src.block, src.dtype == SZX_F32 ? 4 : 8);
                h.total_bytes = src.bytes;
                need = src.n * (src.dtype == SZX_F32 ? 4 : 8);
            }
            uint64_t off;
            if (!s->alloc(need, &off)) {
                if (!running) {
                    result = SZX_ERR_NOMEM;  // it can never fit
                    r.status = SZX_ERR_NOMEM;
                    r.admit_s = r.done_s = now();
                    done[i] = 1;
                    waiting.pop_front();
                    continue;
                }
                break;  // wait for a completion to free memory
            }
            const int slot = idle.back();
            idle.pop_back();
            cudaStream_t st = s->streams[slot];
            szx_status ls;
            if (r.kind == SZX_REQ_COMPRESS) {
                s->h_results[2 * slot] = 0;
                s->h_results[2 * slot + 1] = (uint64_t)SZX_ERR_CUDA;
                // the slots' streams run at once: each call clears its words
                // with a memset node rather than a kernel (Clear::memset)
                ls = compress_async_with(r.d_in, r.n, r.dtype, r.eb, r.block, s->pool + off, granules(need),
                                         s->d_results + 2 * slot, (szx_stream_t)st, Clear::memset);
            } else {
                const szx_request &src = reqs[r.source];
                ls = decompress_async_with(s->pool + src.offset, src.bytes, &h, s->pool + off, need,
                                           s->d_status + slot, (szx_stream_t)st, Clear::memset);
                if (ls == SZX_OK &&
                    cudaMemcpyAsync(s->h_status + slot, s->d_status + slot, sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    ls = SZX_ERR_CUDA;
            }
            if (ls == SZX_OK && cudaEventRecord(s->events[slot], st) != cudaSuccess) ls = SZX_ERR_CUDA;
            waiting.pop_front();
            r.admit_s = now();
            if (ls != SZX_OK) {
                // not launched (host-side argument error): done at once
                s->release(off, need);
                r.status = ls;
                r.done_s = r.admit_s;
                done[i] = 1;
                idle.push_back(slot);
                continue;
            }
            slot_req[slot] = i;
            slot_off[slot] = off;
            slot_need[slot] = need;
            ++running;
            if (running > peak) peak = running;
        }
        // nothing runs, yet the oldest request could not start: nothing will
        // change that, so it fails (this keeps the loop from spinning)
        if (!running && !waiting.empty()) {
            szx_request &r = reqs[waiting.front()];
            r.status = SZX_ERR_INVALID;
            r.admit_s = r.done_s = now();
            done[waiting.front()] = 1;
            waiting.pop_front();
        }
    }
    if (max_in_flight) *max_in_flight = peak;
    return result;
}

void szx_server_destroy(szx_server *s) {
    if (!s) return;
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    if (s->h_results) cudaFreeHost(s->h_results);
    if (s->h_status) cudaFreeHost(s->h_status);
    if (s->d_status) cudaFree(s->d_status);
    delete s;
}

}  // extern "C"
