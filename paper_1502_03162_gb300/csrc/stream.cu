// stream.cu -- block streaming with continuous batching (partitioned time-domain
// convolution: Sec. IV-G notes that direct convolution split into blocks adds no latency and
// needs no extra memory), on the factorized filters of Eqs. 1-2.
//
// Requests (one source each) are admitted into slots while a device pool has room; their
// samples are uploaded on a copy stream that overlaps the rendering, and a source admitted
// before step n joins step n (the step waits for the upload on the GPU).  Sources sharing a
// session id are mixed into that session's stereo stream.  Each step renders one block of B
// samples for every active session with one launch of a captured CUDA graph: one kernel that
// reads the step descriptor from host-mapped memory, and for each session (one CTA, B
// threads, sources in a fixed order)
//   z_e[t]   = sum_src sum_k w_{d,e,k} y[pos + t - i_{d,e,k}]      (reflection taps, Eq. 2)
//   out_e[t] = sum_{l < Lf} f_e[l] z_e[t - l]                       (resonance, state carried)
// and writes the block to host-mapped memory.  A session's arithmetic does not depend on any
// other session, so its output is the same whether it runs alone or in a full batch.  A
// source stays active until its reflection and resonance tails (H - 1 samples) have been
// emitted.
#include <algorithm>
#include <map>
#include <unordered_map>

#include "api_internal.h"

using namespace hrir;
using namespace hrir_host;

namespace {

constexpr int kMaxLf = 64;

struct StepRow {        // one session in a step
    int slot_begin;     // first entry in the slot list
    int slot_count;
    int state;          // resonance-state index
    int fresh;          // 1: the session starts this step (its state is zero)
};

struct StepSlot {       // one source in a step
    int64_t pool_off;   // element offset of the source in the pool
    int64_t len;
    int64_t pos;        // first sample of this block (relative to the source start)
    int dir;
    int pad;
};

struct StepHeader {
    int n_rows;
    int pad[3];
};

struct StreamArgs {
    const StepHeader *hdr;     // host-mapped
    const StepRow *rows;       // host-mapped
    const StepSlot *slots;     // host-mapped
    const float *pool;
    const uint16_t *tap_idx;   // [n_dirs][2][k_max]
    const float *tap_w;
    const uint8_t *tap_nnz;
    int k_max;
    int n_dirs;
    const float *res;          // [2][Lf]
    int res_len;
    float *state;              // [max_slots][2][kMaxLf - 1]
    float *out;                // host-mapped [max_slots][2][B]
    int block;
    int *status;
};

__global__ void __launch_bounds__(256) stream_step_kernel(const StreamArgs a)
{
    __shared__ float zs[2][kMaxLf - 1 + 256];
    __shared__ float fs[2][kMaxLf];
    const int t = threadIdx.x;
    const int B = a.block;
    const int lf = a.res_len;
    const int n_rows = a.hdr->n_rows;
    for (int i = t; i < 2 * lf; i += blockDim.x) fs[i / lf][i % lf] = a.res[i];
    for (int row = blockIdx.x; row < n_rows; row += gridDim.x) {
        const StepRow r = a.rows[row];
        float z[2] = {0.f, 0.f};
        if (t < B) {
            for (int j = 0; j < r.slot_count; ++j) {
                const StepSlot sl = a.slots[r.slot_begin + j];
                const int d = sl.dir;
                if ((unsigned)d >= (unsigned)a.n_dirs) {
                    if (t == 0) atomicOr(a.status, DEV_BAD_DIR);
                    continue;
                }
                const float *y = a.pool + sl.pool_off;
                for (int e = 0; e < 2; ++e) {
                    const size_t row_t = ((size_t)d * 2 + e) * a.k_max;
                    const int k = a.tap_nnz[(size_t)d * 2 + e];
                    float acc = z[e];
                    for (int q = 0; q < k; ++q) {
                        const int64_t n = sl.pos + t - (int64_t)a.tap_idx[row_t + q];
                        const float v = (n >= 0 && n < sl.len) ? __ldg(y + n) : 0.f;
                        acc = fmaf(a.tap_w[row_t + q], v, acc);
                    }
                    z[e] = acc;
                }
            }
        }
        float *st = a.state + (size_t)r.state * 2 * (kMaxLf - 1);
        __syncthreads();
        for (int i = t; i < 2 * (lf - 1); i += blockDim.x) {
            const int e = i / (lf - 1), l = i % (lf - 1);
            zs[e][l] = r.fresh ? 0.f : st[e * (kMaxLf - 1) + l];
        }
        if (t < B) {
            zs[0][lf - 1 + t] = z[0];
            zs[1][lf - 1 + t] = z[1];
        }
        __syncthreads();
        if (t < B) {
            float *o = a.out + (size_t)row * 2 * B;
            for (int e = 0; e < 2; ++e) {
                float acc = 0.f;
                for (int l = 0; l < lf; ++l) acc = fmaf(fs[e][l], zs[e][lf - 1 + t - l], acc);
                o[e * B + t] = acc;
            }
        }
        // carry the last Lf - 1 reflection outputs to the next block
        for (int i = t; i < 2 * (lf - 1); i += blockDim.x) {
            const int e = i / (lf - 1), l = i % (lf - 1);
            st[e * (kMaxLf - 1) + l] = zs[e][B + l];
        }
        __syncthreads();
    }
}

// First-fit allocator over the device pool (element offsets, 64-element granules).
struct PoolAlloc {
    std::map<int64_t, int64_t> free_;  // offset -> size
    int64_t used = 0;
    void reset(int64_t n)
    {
        free_.clear();
        if (n > 0) free_[0] = n;
        used = 0;
    }
    int64_t alloc(int64_t n)
    {
        n = (n + 63) / 64 * 64;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const int64_t off = it->first, rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                used += n;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t n)
    {
        n = (n + 63) / 64 * 64;
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Slot {
    bool used = false;
    bool ready = false;       // upload finished
    int64_t req_id = 0, session = 0;
    int64_t pool_off = 0, len = 0, pos = 0;
    int dir = 0;
    cudaEvent_t uploaded = nullptr;
};

struct Session {
    int state = -1;
    int live_slots = 0;
    bool fresh = true;
};

}  // namespace

struct hrir_stream {
    int block = 0, max_slots = 0;
    cudaStream_t st = nullptr, copy_st = nullptr;
    float *pool = nullptr;
    int64_t pool_elems = 0;
    PoolAlloc alloc;
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    std::map<int64_t, Session> sessions;      // ordered: deterministic row order
    std::vector<int> free_states;
    float *state = nullptr;
    // host-mapped step descriptor and output
    StepHeader *h_hdr = nullptr;
    StepRow *h_rows = nullptr;
    StepSlot *h_slots = nullptr;
    float *h_out = nullptr;
    std::vector<int64_t> row_sessions;
    std::vector<int> order;                   // used slots in (session, slot) order
    std::vector<int> pending;                 // admitted since the last step (upload in flight)
    int *h_status = nullptr;                  // status word after each step (page-locked)
    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_def = nullptr;
};

namespace {

void stream_free(hrir_stream *s)
{
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->copy_st) cudaStreamSynchronize(s->copy_st);
    for (auto &sl : s->slots)
        if (sl.uploaded) cudaEventDestroy(sl.uploaded);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->graph_def) cudaGraphDestroy(s->graph_def);
    cudaFree(s->pool);
    cudaFree(s->state);
    cudaFreeHost(s->h_hdr);
    cudaFreeHost(s->h_rows);
    cudaFreeHost(s->h_slots);
    cudaFreeHost(s->h_out);
    cudaFreeHost(s->h_status);
    if (s->copy_st) cudaStreamDestroy(s->copy_st);
    delete s;
}

}  // namespace

extern "C" {

int hrir_stream_close(hrir_ctx *ctx)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    stream_free(ctx->stream);
    ctx->stream = nullptr;
    return HRIR_OK;
}

int hrir_stream_open(hrir_ctx *ctx, int block, int max_slots, size_t pool_bytes, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded");
    if (block != 128 && block != 256) return fail(ctx, HRIR_EINVAL, "block must be 128 or 256");
    if (max_slots < 1 || max_slots > (1 << 16)) return fail(ctx, HRIR_EINVAL, "max_slots out of range");
    if (ctx->res_len > kMaxLf) return fail(ctx, HRIR_EINVAL, "streaming supports Lf <= %d", kMaxLf);
    if (pool_bytes < 4096) return fail(ctx, HRIR_EINVAL, "pool_bytes too small");
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    hrir_stream_close(ctx);
    hrir_stream *s = new hrir_stream();
    s->block = block;
    s->max_slots = max_slots;
    s->st = (cudaStream_t)stream;
    s->pool_elems = (int64_t)(pool_bytes / sizeof(float));
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaMalloc(&s->pool, (size_t)s->pool_elems * sizeof(float))) != cudaSuccess) break;
        if ((e = cudaMalloc(&s->state, (size_t)max_slots * 2 * (kMaxLf - 1) * sizeof(float))) != cudaSuccess)
            break;
        if ((e = cudaHostAlloc(&s->h_hdr, sizeof(StepHeader), cudaHostAllocMapped)) != cudaSuccess) break;
        if ((e = cudaHostAlloc(&s->h_rows, (size_t)max_slots * sizeof(StepRow), cudaHostAllocMapped)) != cudaSuccess)
            break;
        if ((e = cudaHostAlloc(&s->h_slots, (size_t)max_slots * sizeof(StepSlot), cudaHostAllocMapped)) != cudaSuccess)
            break;
        if ((e = cudaHostAlloc(&s->h_out, (size_t)max_slots * 2 * block * sizeof(float), cudaHostAllocMapped)) !=
            cudaSuccess)
            break;
        if ((e = cudaHostAlloc(&s->h_status, sizeof(int), cudaHostAllocDefault)) != cudaSuccess) break;
    } while (0);
    if (e != cudaSuccess) {
        stream_free(s);
        cudaGetLastError();
        return fail(ctx, e == cudaErrorMemoryAllocation ? HRIR_ENOMEM : HRIR_ECUDA,
                    "stream allocation failed: %s", cudaGetErrorString(e));
    }
    s->alloc.reset(s->pool_elems);
    s->slots.resize(max_slots);
    for (int i = max_slots - 1; i >= 0; --i) {
        s->free_slots.push_back(i);
        s->free_states.push_back(i);
    }
    s->h_hdr->n_rows = 0;

    // Capture the step: one kernel node with device views of the mapped descriptor/output,
    // then the status word copied to page-locked host memory (read after the step's sync).
    StreamArgs a;
    void *p = nullptr;
    cudaHostGetDevicePointer(&p, s->h_hdr, 0);
    a.hdr = static_cast<const StepHeader *>(p);
    cudaHostGetDevicePointer(&p, s->h_rows, 0);
    a.rows = static_cast<const StepRow *>(p);
    cudaHostGetDevicePointer(&p, s->h_slots, 0);
    a.slots = static_cast<const StepSlot *>(p);
    cudaHostGetDevicePointer(&p, s->h_out, 0);
    a.out = static_cast<float *>(p);
    a.pool = s->pool;
    a.tap_idx = ctx->d_tap_idx;
    a.tap_w = ctx->d_tap_w;
    a.tap_nnz = ctx->d_tap_nnz;
    a.k_max = ctx->k_max > 0 ? ctx->k_max : 1;
    a.n_dirs = ctx->n_dirs;
    a.res = ctx->d_res;
    a.res_len = ctx->res_len;
    a.state = s->state;
    a.block = block;
    a.status = ctx->d_status;
    const int grid = std::min(max_slots, ctx->num_sms * 8);
    cudaStream_t cap = nullptr;
    do {
        if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        stream_step_kernel<<<grid, 256, 0, cap>>>(a);
        if ((e = cudaMemcpyAsync(s->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, cap)) !=
            cudaSuccess) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cap, &g);
            if (g) cudaGraphDestroy(g);
            break;
        }
        if ((e = cudaStreamEndCapture(cap, &s->graph_def)) != cudaSuccess) break;
        e = cudaGraphInstantiate(&s->graph, s->graph_def, 0);
    } while (0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        stream_free(s);
        cudaGetLastError();
        return fail(ctx, HRIR_ECUDA, "step graph capture failed: %s", cudaGetErrorString(e));
    }
    ctx->stream = s;
    return HRIR_OK;
}

int hrir_stream_admit(hrir_ctx *ctx, int64_t req_id, int64_t session, const float *host_src,
                      int64_t len, int dir)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    hrir_stream *s = ctx->stream;
    if (!s) return fail(ctx, HRIR_ESTATE, "no stream open");
    if (len < 1 || !host_src) return fail(ctx, HRIR_EINVAL, "empty source");
    if (dir < 0 || dir >= ctx->n_dirs) return fail(ctx, HRIR_EINVAL, "direction %d out of range", dir);
    if (s->free_slots.empty()) return fail(ctx, HRIR_EBUSY, "all %d slots busy", s->max_slots);
    auto sit = s->sessions.find(session);
    if (sit == s->sessions.end() && s->free_states.empty())
        return fail(ctx, HRIR_EBUSY, "no free session state");
    const int64_t off = s->alloc.alloc(len);
    if (off < 0) return fail(ctx, HRIR_ENOMEM, "pool full (%lld of %lld elements used)",
                             (long long)s->alloc.used, (long long)s->pool_elems);
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int id = s->free_slots.back();
    Slot &sl = s->slots[id];
    if (!sl.uploaded) {
        if (cudaEventCreateWithFlags(&sl.uploaded, cudaEventDisableTiming) != cudaSuccess) {
            s->alloc.release(off, len);
            return fail(ctx, HRIR_ECUDA, "event creation failed");
        }
    }
    cudaError_t e = cudaMemcpyAsync(s->pool + off, host_src, (size_t)len * sizeof(float),
                                    cudaMemcpyHostToDevice, s->copy_st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.uploaded, s->copy_st);
    if (e != cudaSuccess) {
        s->alloc.release(off, len);
        return fail(ctx, HRIR_ECUDA, "upload failed: %s", cudaGetErrorString(e));
    }
    s->free_slots.pop_back();
    sl.used = true;
    sl.ready = false;
    sl.req_id = req_id;
    sl.session = session;
    sl.pool_off = off;
    sl.len = len;
    sl.pos = 0;
    sl.dir = dir;
    if (sit == s->sessions.end()) {
        Session ss;
        ss.state = s->free_states.back();
        s->free_states.pop_back();
        sit = s->sessions.emplace(session, ss).first;
    }
    sit->second.live_slots += 1;
    // keep the step order (session, slot): insert the new slot at its place
    const auto before = [&](int x, int y) {
        return s->slots[x].session != s->slots[y].session ? s->slots[x].session < s->slots[y].session : x < y;
    };
    s->order.insert(std::lower_bound(s->order.begin(), s->order.end(), id, before), id);
    s->pending.push_back(id);
    return HRIR_OK;
}

int hrir_stream_step(hrir_ctx *ctx, const float **out_blocks, const int64_t **out_sessions, int *n_out,
                     int64_t *done_ids, int *n_done)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    hrir_stream *s = ctx->stream;
    if (!s) return fail(ctx, HRIR_ESTATE, "no stream open");
    if (!out_blocks || !out_sessions || !n_out || !n_done)
        return fail(ctx, HRIR_EINVAL, "NULL output pointer");
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int64_t tail = ctx->hrir_len - 1;
    // sources admitted since the last step join this one; the step's kernel waits on the GPU
    // for their uploads (the host does not block)
    for (int id : s->pending) {
        HRIR_CUDA_TRY(ctx, cudaStreamWaitEvent(s->st, s->slots[id].uploaded, 0));
        s->slots[id].ready = true;
    }
    s->pending.clear();
    // descriptor: sessions in id order, each session's sources in slot order (the order kept
    // by hrir_stream_admit)
    s->row_sessions.clear();
    int n_rows = 0;
    const int n_sl = (int)s->order.size();
    for (int j = 0; j < n_sl; ++j) {
        const Slot &sl = s->slots[s->order[j]];
        StepSlot &d = s->h_slots[j];
        d.pool_off = sl.pool_off;
        d.len = sl.len;
        d.pos = sl.pos;
        d.dir = sl.dir;
        d.pad = 0;
        if (j == 0 || s->slots[s->order[j - 1]].session != sl.session) {
            Session &ss = s->sessions[sl.session];
            StepRow &r = s->h_rows[n_rows++];
            r.slot_begin = j;
            r.slot_count = 0;
            r.state = ss.state;
            r.fresh = ss.fresh ? 1 : 0;
            ss.fresh = false;
            s->row_sessions.push_back(sl.session);
        }
        s->h_rows[n_rows - 1].slot_count += 1;
    }
    s->h_hdr->n_rows = n_rows;
    if (n_rows > 0) {
        HRIR_CUDA_TRY(ctx, cudaGraphLaunch(s->graph, s->st));
        HRIR_CUDA_TRY(ctx, cudaStreamSynchronize(s->st));
    }
    // advance; retire sources whose tails are out, and sessions without sources
    int nd = 0;
    size_t kept = 0;
    for (size_t j = 0; j < s->order.size(); ++j) {
        const int i = s->order[j];
        Slot &sl = s->slots[i];
        sl.pos += s->block;
        if (sl.pos >= sl.len + tail) {
            if (done_ids) done_ids[nd] = sl.req_id;
            ++nd;
            s->alloc.release(sl.pool_off, sl.len);
            sl.used = false;
            s->free_slots.push_back(i);
            auto it = s->sessions.find(sl.session);
            if (--it->second.live_slots == 0) {
                s->free_states.push_back(it->second.state);
                s->sessions.erase(it);
            }
        } else {
            s->order[kept++] = i;
        }
    }
    s->order.resize(kept);
    *out_blocks = s->h_out;
    *out_sessions = s->row_sessions.data();
    *n_out = n_rows;
    *n_done = nd;
    if (n_rows > 0) {
        const int st = *s->h_status;          // copied by the step's graph
        if (st) {
            HRIR_CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
            return fail(ctx, HRIR_EINVAL, "a direction id was out of range (rendered as silence)");
        }
    }
    return HRIR_OK;
}

int hrir_stream_stats(hrir_ctx *ctx, int *active, int *pending, int64_t *pool_used_bytes)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    hrir_stream *s = ctx->stream;
    if (!s) return fail(ctx, HRIR_ESTATE, "no stream open");
    int a = 0, p = 0;
    for (const auto &sl : s->slots) {
        if (!sl.used) continue;
        if (sl.ready) ++a;
        else ++p;
    }
    if (active) *active = a;
    if (pending) *pending = p;
    if (pool_used_bytes) *pool_used_bytes = s->alloc.used * (int64_t)sizeof(float);
    return HRIR_OK;
}

}  // extern "C"
