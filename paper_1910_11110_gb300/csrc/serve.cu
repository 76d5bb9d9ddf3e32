// serve.cu -- continuous batching of check requests on one GPU.
//
// A server owns a device memory pool (the budget), max_slots CUDA streams and
// a worker thread.  Requests are copied at submission and queued.  The worker
// admits queued requests in arrival order whenever a slot is free, the pool
// can hold the request's buffers, and the request's session has nothing in
// flight (a session's requests see each other's statuses, so they run in
// submission order; different sessions overlap on the device).  Each admitted
// request runs on its slot's stream: inputs are staged through pinned memory
// and copied to the device, the trace kernel (or the relation-mode kernel for
// a program) runs with the session's status table as initial and final status,
// the per-op results come back to pinned memory, and an event marks the end.
// The worker polls those events, hands results to amc_serve_poll, and frees
// the slot and the request's pool space, which may admit the next requests.
// A session's table stays on the device between requests and holds, per
// variable, the SET of statuses it may have (a status mask), so that trace and
// program requests can follow one another in a session.  Until the session has
// run a program with an If or While every set is a singleton: a trace request
// is then checked by the trace kernels on status codes (the table converted to
// codes and back) and reports codes; after such a program a trace request is
// checked in relation mode as a straight-line program and reports masks.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "amc_internal.cuh"
#include "batch.cuh"
#include "scan_trace.cuh"

using namespace amc;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device allocation (offsets, 256-byte granules).
class Pool {
public:
    bool init(size_t bytes, bool pinned_host)
    {
        bytes = align_up(bytes, 256);
        host_ = pinned_host;
        const cudaError_t e = host_ ? cudaHostAlloc(&base_, bytes, cudaHostAllocDefault) : cudaMalloc(&base_, bytes);
        if (e != cudaSuccess) {
            base_ = nullptr;
            return false;
        }
        size_ = bytes;
        free_[0] = bytes;
        return true;
    }
    void release()
    {
        if (base_) host_ ? cudaFreeHost(base_) : cudaFree(base_);
        base_ = nullptr;
    }
    // returns offset or SIZE_MAX
    size_t alloc(size_t n)
    {
        n = align_up(n ? n : 256, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first, sz = it->second;
                free_.erase(it);
                if (sz > n) free_[off + n] = sz - n;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void free(size_t off, size_t n)
    {
        n = align_up(n ? n : 256, 256);
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
    uint8_t* ptr(size_t off) const { return static_cast<uint8_t*>(base_) + off; }
    size_t size() const { return size_; }

private:
    void* base_ = nullptr;
    size_t size_ = 0;
    bool host_ = false;
    std::map<size_t, size_t> free_;
};

struct Session {
    bool known = false;
    bool det = true;                 // every set is a singleton (no If / While program has run)
    int32_t n_vars = 0;
    size_t table_off = SIZE_MAX;     // status masks, n_vars bytes
    bool busy = false;
};

struct Request {
    uint64_t ticket = 0, session = 0;
    int kind = 0;
    int32_t n_vars = 0;
    int64_t n = 0;
    const uint8_t* src_ks = nullptr;   // borrowed inputs (AMC_REQ_BORROW), else staged copies
    const int32_t* src_var = nullptr;
    size_t host_off = SIZE_MAX;      // pinned: op bytes [n], ids [4n] at 256-aligned offsets, results [n], small
    size_t host_bytes = 0;
    int64_t first_fault = -1;
    int error = AMC_OK;
    bool has_struct = false;         // a program with If / While tokens
    int is_mask = 0;                 // the result holds status masks
    int state = 0;                   // 0 queued, 1 running, 2 done
    int slot = -1;
    size_t off = SIZE_MAX, bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::shared_ptr<Request> req;
    bool launching = false;          // the worker is enqueueing its work (outside the lock)
};

// pinned layout of a request: staged inputs (none when borrowed), results,
// and a small block (first fault, error word, program offsets)
struct HostLayout {
    size_t ks, var, out, small, total;
};
HostLayout host_layout(int64_t n, bool borrowed)
{
    HostLayout L;
    L.ks = 0;
    L.var = borrowed ? 0 : align_up((size_t)n, 256);
    L.out = borrowed ? 0 : L.var + align_up(4 * (size_t)n, 256);
    L.small = L.out + align_up((size_t)n, 256);
    L.total = L.small + 256;
    return L;
}

}  // namespace

struct amc_server {
    std::mutex mu;
    std::condition_variable cv;
    Pool pool;                       // device memory: the budget
    Pool host;                       // pinned staging of inputs and results
    cudaStream_t ctl = nullptr;
    std::vector<Slot> slots;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    std::map<uint64_t, Session> sessions;
    std::deque<uint64_t> finished;   // tickets finished since the last amc_serve_completed
    uint64_t next_ticket = 1;
    size_t max_queue = 1 << 20;
    std::atomic<bool> stop{false};
    std::thread worker;
    int device = 0;
    int* err = nullptr;
};

namespace {

// Host-side validation of a request.  A trace is checked on the device by
// the kernels themselves (op bytes, ids; the request's own error word); a
// program's structure is checked here (its constructs decide how it runs).
// *has_struct: the program has If / While tokens.
int validate(const amc_request* r, bool* has_struct)
{
    *has_struct = false;
    if (!r || r->n_items < 0 || r->n_vars < 1 || (r->n_items > 0 && (!r->kind_side || !r->var))) return AMC_E_INVALID;
    if (r->kind != AMC_REQ_TRACE && r->kind != AMC_REQ_PROGRAM) return AMC_E_INVALID;
    if (r->flags & ~AMC_REQ_BORROW) return AMC_E_INVALID;
    if (r->kind == AMC_REQ_TRACE) return r->n_items > INT32_MAX ? AMC_E_RANGE : AMC_OK;
    // programs: op tokens in range, constructs balanced and nested within AMC_MAX_DEPTH
    std::vector<int64_t> ends;
    std::vector<int> kinds;
    for (int64_t i = 0; i < r->n_items; ++i) {
        const uint8_t k = r->kind_side[i];
        if (k & 0xE0) return AMC_E_INVALID;
        const int kk = k & 15;
        if (kk <= AMC_K_PW) {
            if (r->var[i] < 0 || r->var[i] >= r->n_vars) return AMC_E_RANGE;
            continue;
        }
        if (k & 0x10) return AMC_E_INVALID;
        if (kk == AMC_T_IF || kk == AMC_T_WHILE) {
            *has_struct = true;
            const int64_t len = r->var[i];
            if (len < 0 || (int)ends.size() >= AMC_MAX_DEPTH) return AMC_E_INVALID;
            int64_t end;
            if (kk == AMC_T_IF) {
                const int64_t e = i + 1 + len;
                if (e >= r->n_items || r->kind_side[e] != AMC_T_ELSE || r->var[e] < 0) return AMC_E_INVALID;
                end = e + 1 + r->var[e];
            } else {
                end = i + 1 + len;
            }
            if (end >= r->n_items || r->kind_side[end] != AMC_T_END) return AMC_E_INVALID;
            if (!ends.empty() && end >= ends.back()) return AMC_E_INVALID;
            ends.push_back(end);
            kinds.push_back(kk);
        } else if (kk == AMC_T_ELSE) {
            if (ends.empty() || kinds.back() != AMC_T_IF) return AMC_E_INVALID;
        } else if (kk == AMC_T_END) {
            if (ends.empty() || ends.back() != i) return AMC_E_INVALID;
            ends.pop_back();
            kinds.pop_back();
        } else {
            return AMC_E_INVALID;
        }
    }
    return ends.empty() ? AMC_OK : AMC_E_INVALID;
}

size_t request_bytes(const Request& r)
{
    const size_t n = (size_t)r.n;
    size_t b = align_up(n, 256) + align_up(4 * n, 256) + align_up(n, 256) + 512;   // ks, var, out, small
    // relation mode, one program, never split; construct rows only when the
    // request has constructs
    size_t w = batch_workspace_bytes(r.n, 1, true, r.has_struct ? AMC_MAX_DEPTH : 0) + 256;
    if (r.kind == AMC_REQ_TRACE) {
        // trace kernels: workspace, first faults, the session's statuses as
        // codes; for sessions of status sets also one pass's statuses, the
        // final sets and the passes' first faults
        const size_t t = scan_workspace_bytes(r.n, r.n_vars) + align_up(4 * (size_t)r.n_vars, 256) +
                         align_up((size_t)r.n_vars, 256) + align_up(n, 256) + align_up((size_t)r.n_vars, 256) + 256;
        if (t > w) w = t;
    }
    return b + w;
}

// A straight-line trace over status sets (Section 3.2's semantics on every
// member of the entry set, as relation mode computes it): each op is a
// function of the status, so the set after a prefix is the image of the entry
// set, the union of the members' trajectories.  Pass k checks the trace from
// the k-th member of every variable's set (its last member when the set has
// fewer); the step sets, final sets and first fault are the union / minimum
// over the five passes.  Sets are never empty (every op maps a status to a
// status).
constexpr int SET_PASSES = 5;

__global__ void member_codes_kernel(const uint8_t* __restrict__ m, uint8_t* __restrict__ c, int32_t n, int k)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint32_t x = m[v] & 31u, pick = 0;
    for (int j = 0; x; ++j, x &= x - 1) {
        pick = (uint32_t)(__ffs(x) - 1);
        if (j == k) break;
    }
    c[v] = (uint8_t)pick;
}

// out[i] |= 1 << step[i] (the first pass sets out[i]); the same for the
// final sets; *ff = min over the passes
__global__ void merge_pass_kernel(const uint8_t* __restrict__ step, uint8_t* __restrict__ out, int64_t n,
                                  const uint8_t* __restrict__ fin, uint8_t* __restrict__ fset, int32_t nv,
                                  const int64_t* __restrict__ ff_pass, int64_t* __restrict__ ff, int first)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint8_t b = (uint8_t)(1u << (step[i] & 7u));
        out[i] = first ? b : (uint8_t)(out[i] | b);
    }
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        const uint8_t b = (uint8_t)(1u << (fin[v] & 7u));
        fset[v] = first ? b : (uint8_t)(fset[v] | b);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t a = *ff_pass, cur = first ? -1 : *ff;
        *ff = a < 0 ? cur : (cur < 0 || a < cur ? a : cur);
    }
}

__global__ void copy_sets_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, int32_t n)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) dst[v] = src[v];
}

// singleton masks <-> status codes
__global__ void masks_to_codes_kernel(const uint8_t* __restrict__ m, uint8_t* __restrict__ c, int32_t n)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) c[v] = (uint8_t)(__ffs(m[v]) - 1);
}
__global__ void codes_to_masks_kernel(const uint8_t* __restrict__ c, uint8_t* __restrict__ m, int32_t n)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) m[v] = (uint8_t)(1u << (c[v] & 7u));
}

// Launch an admitted request on its slot (worker thread, lock held).
int launch(amc_server* s, Slot& sl, Request& r, Session& ses)
{
    const size_t n = (size_t)r.n;
    const HostLayout H = host_layout(r.n, r.src_ks != nullptr);
    uint8_t* h = s->host.ptr(r.host_off);
    uint8_t* d = s->pool.ptr(r.off);
    uint8_t* d_ks = d;
    int32_t* d_var = reinterpret_cast<int32_t*>(d + align_up(n, 256));
    uint8_t* d_out = d + align_up(n, 256) + align_up(4 * n, 256);
    int64_t* d_small = reinterpret_cast<int64_t*>(d_out + align_up(n, 256));
    uint8_t* d_ws = reinterpret_cast<uint8_t*>(d_small) + 512;
    uint8_t* table = s->pool.ptr(ses.table_off);
    cudaStream_t st = sl.stream;
    if (n) {
        const uint8_t* ks = r.src_ks ? r.src_ks : h + H.ks;
        const void* vs = r.src_var ? static_cast<const void*>(r.src_var) : static_cast<const void*>(h + H.var);
        if (cudaMemcpyAsync(d_ks, ks, n, cudaMemcpyHostToDevice, st) != cudaSuccess) return AMC_E_CUDA;
        if (cudaMemcpyAsync(d_var, vs, 4 * n, cudaMemcpyHostToDevice, st) != cudaSuccess) return AMC_E_CUDA;
    }
    int64_t* d_ff = d_small;
    int* d_err = reinterpret_cast<int*>(d_small + 7);      // this request's device-side error word
    if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) return AMC_E_CUDA;
    int rc;
    const unsigned vb = (unsigned)((r.n_vars + 255) / 256);
    if (r.kind == AMC_REQ_TRACE && ses.det) {
        // every set is a singleton: the trace kernels on status codes
        uint8_t* codes = d_ws + scan_workspace_bytes(r.n, r.n_vars) + align_up(4 * (size_t)r.n_vars, 256);
        masks_to_codes_kernel<<<vb, 256, 0, st>>>(table, codes, r.n_vars);
        ScanLaunch L;
        L.kind_side = d_ks;
        L.var = d_var;
        L.n_ops = r.n;
        L.n_vars = r.n_vars;
        L.init = codes;
        L.step = d_out;
        L.final_status = codes;           // in place: read and written per variable by one thread
        L.vff = reinterpret_cast<int32_t*>(d_ws + scan_workspace_bytes(r.n, r.n_vars));
        L.first_fault = d_ff;
        L.err = d_err;
        L.workspace = d_ws;
        rc = launch_scan_trace(L, st);
        if (!rc) codes_to_masks_kernel<<<vb, 256, 0, st>>>(codes, table, r.n_vars);
        r.is_mask = 0;
    } else if (r.kind == AMC_REQ_TRACE) {
        // a trace over sets of several statuses: one trace check per member
        uint8_t* after = d_ws + scan_workspace_bytes(r.n, r.n_vars);
        int32_t* vff = reinterpret_cast<int32_t*>(after);
        uint8_t* codes = after + align_up(4 * (size_t)r.n_vars, 256);
        uint8_t* step_k = codes + align_up((size_t)r.n_vars, 256);
        uint8_t* fset = step_k + align_up(n, 256);
        int64_t* ff_k = reinterpret_cast<int64_t*>(fset + align_up((size_t)r.n_vars, 256));
        const unsigned mb = (unsigned)((n > (size_t)r.n_vars ? n : (size_t)r.n_vars) + 255) / 256;
        const unsigned mgrid = mb < 4096 ? (mb ? mb : 1) : 4096;
        rc = AMC_OK;
        for (int k = 0; k < SET_PASSES && !rc; ++k) {
            member_codes_kernel<<<vb, 256, 0, st>>>(table, codes, r.n_vars, k);
            ScanLaunch L;
            L.kind_side = d_ks;
            L.var = d_var;
            L.n_ops = r.n;
            L.n_vars = r.n_vars;
            L.init = codes;
            L.step = step_k;
            L.final_status = codes;       // in place, as above
            L.vff = vff;
            L.first_fault = ff_k;
            L.err = d_err;
            L.workspace = d_ws;
            rc = launch_scan_trace(L, st);
            if (!rc)
                merge_pass_kernel<<<mgrid, 256, 0, st>>>(step_k, d_out, (int64_t)n, codes, fset, r.n_vars, ff_k, d_ff,
                                                         k == 0);
        }
        if (!rc) copy_sets_kernel<<<vb, 256, 0, st>>>(fset, table, r.n_vars);
        r.is_mask = 1;
    } else {
        // a program: token offsets {0, n}, var offsets {0, n_vars}, n_vars
        int64_t* hs = reinterpret_cast<int64_t*>(h + H.small);
        hs[1] = 0;
        hs[2] = (int64_t)r.n;
        hs[3] = 0;
        hs[4] = (int64_t)r.n_vars;
        reinterpret_cast<int32_t*>(hs + 5)[0] = r.n_vars;
        if (cudaMemcpyAsync(d_small + 1, hs + 1, 5 * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return AMC_E_CUDA;
        BatchLaunch B;
        B.tok = d_ks;
        B.payload = d_var;
        B.prog_tok_off = d_small + 1;
        B.prog_var_off = d_small + 3;
        B.prog_nvars = reinterpret_cast<const int32_t*>(d_small + 5);
        B.n_progs = 1;
        B.n_tokens = r.n;
        B.init_mask = table;
        B.step_mask = d_out;
        B.final_mask = table;
        B.prog_first_fault = d_ff;
        B.err = d_err;
        B.workspace = d_ws;
        B.longest_first = 0;
        B.no_split = 1;
        B.save_rows = r.has_struct ? AMC_MAX_DEPTH : 0;
        rc = launch_batch(B, st);
        r.is_mask = 1;
        if (r.has_struct) ses.det = false;      // later requests see sets of several statuses
    }
    if (rc) return rc;
    if (n && cudaMemcpyAsync(h + H.out, d_out, n, cudaMemcpyDeviceToHost, st) != cudaSuccess) return AMC_E_CUDA;
    if (cudaMemcpyAsync(h + H.small, d_ff, 64, cudaMemcpyDeviceToHost, st) != cudaSuccess) return AMC_E_CUDA;
    if (cudaEventRecord(sl.done, st) != cudaSuccess) return AMC_E_CUDA;
    return AMC_OK;
}

void finish(amc_server* s, Slot& sl)
{
    Request& r = *sl.req;
    const uint8_t* small = s->host.ptr(r.host_off) + host_layout(r.n, r.src_ks != nullptr).small;
    memcpy(&r.first_fault, small, 8);
    int e = 0;
    memcpy(&e, small + 56, sizeof(int));
    if (e) r.error = e;
    r.t_done = now_s();
    r.state = 2;
    s->pool.free(r.off, r.bytes);
    s->sessions[r.session].busy = false;
    s->finished.push_back(r.ticket);
    sl.req.reset();
}

// The worker: under the lock it retires finished slots and admits queued
// requests (memory, slot, session); it enqueues their copies and kernels with
// the lock released, so that submit and poll never wait for CUDA calls.
void worker_loop(amc_server* s)
{
    cudaSetDevice(s->device);
    std::vector<Slot*> batch;
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        bool progress = false;
        bool running = false;
        for (Slot& sl : s->slots) {
            if (!sl.req || sl.launching) continue;
            running = true;
            if (cudaEventQuery(sl.done) == cudaSuccess) {
                finish(s, sl);
                progress = true;
            }
        }
        // admission in arrival order; a request waits if its session is busy
        batch.clear();
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Slot* free_slot = nullptr;
            for (Slot& sl : s->slots)
                if (!sl.req) { free_slot = &sl; break; }
            if (!free_slot) break;
            Request& r = **it;
            Session& ses = s->sessions[r.session];
            if (ses.busy) { ++it; continue; }
            const size_t off = s->pool.alloc(r.bytes);
            if (off == SIZE_MAX) break;                     // wait for memory
            r.off = off;
            r.t_admit = now_s();
            r.state = 1;
            ses.busy = true;
            free_slot->req = *it;
            free_slot->launching = true;
            batch.push_back(free_slot);
            it = s->queue.erase(it);
            progress = true;
            running = true;
        }
        if (!batch.empty()) {
            // sessions and requests of admitted slots are touched by no one
            // else until their slot is retired
            std::vector<std::pair<Request*, Session*>> work;
            for (Slot* sl : batch) work.emplace_back(sl->req.get(), &s->sessions[sl->req->session]);
            lock.unlock();
            std::vector<int> rcs(batch.size());
            for (size_t k = 0; k < batch.size(); ++k) rcs[k] = launch(s, *batch[k], *work[k].first, *work[k].second);
            lock.lock();
            for (size_t k = 0; k < batch.size(); ++k) {
                Slot& sl = *batch[k];
                sl.launching = false;
                if (rcs[k]) {
                    cudaStreamSynchronize(sl.stream);
                    Request& r = *sl.req;
                    r.error = rcs[k];
                    r.t_done = now_s();
                    r.state = 2;
                    s->pool.free(r.off, r.bytes);
                    s->sessions[r.session].busy = false;
                    s->finished.push_back(r.ticket);
                    sl.req.reset();
                }
            }
        }
        if (s->stop && s->queue.empty() && !running) break;
        if (!progress) {
            if (running)
                s->cv.wait_for(lock, std::chrono::microseconds(20));
            else
                s->cv.wait_for(lock, std::chrono::milliseconds(2));
        }
    }
}

}  // namespace

extern "C" {

int amc_server_create(size_t mem_budget_bytes, int max_slots, amc_server** out)
{
    if (!out || max_slots < 1 || max_slots > 256 || mem_budget_bytes < (1u << 20)) return AMC_E_INVALID;
    std::unique_ptr<amc_server> s(new amc_server());
    if (cudaGetDevice(&s->device) != cudaSuccess) return AMC_E_CUDA;
    s->err = device_error_word();
    if (!s->err) return AMC_E_CUDA;
    if (!s->pool.init(mem_budget_bytes, false)) return AMC_E_NOMEM;
    const size_t host_bytes = mem_budget_bytes < ((size_t)4 << 30) ? mem_budget_bytes : ((size_t)4 << 30);
    if (!s->host.init(host_bytes, true)) {
        s->pool.release();
        return AMC_E_NOMEM;
    }
    if (cudaStreamCreateWithFlags(&s->ctl, cudaStreamNonBlocking) != cudaSuccess) return AMC_E_CUDA;
    s->slots.resize(max_slots);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) return AMC_E_CUDA;
        if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) return AMC_E_CUDA;
    }
    amc_server* raw = s.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return AMC_OK;
}

int amc_serve_submit(amc_server* s, uint64_t session_id, const amc_request* req, uint64_t* ticket)
{
    if (!s || !ticket) return AMC_E_INVALID;
    bool has_struct = false;
    const int v = validate(req, &has_struct);
    if (v) return v;
    auto r = std::make_shared<Request>();
    r->has_struct = has_struct;
    r->session = session_id;
    r->kind = req->kind;
    r->n_vars = req->n_vars;
    r->n = req->n_items;
    r->bytes = request_bytes(*r);
    const bool borrowed = (req->flags & AMC_REQ_BORROW) != 0;
    if (borrowed) {
        r->src_ks = req->kind_side;
        r->src_var = req->var;
    }
    const HostLayout H = host_layout(r->n, borrowed);
    r->host_bytes = H.total;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->queue.size() >= s->max_queue) return AMC_E_AGAIN;
    Session& ses = s->sessions[session_id];
    if (ses.known && ses.n_vars != req->n_vars) return AMC_E_INVALID;   // sized by its first request
    if (r->bytes + align_up((size_t)req->n_vars, 256) > s->pool.size() || H.total > s->host.size())
        return AMC_E_NOMEM;
    r->host_off = s->host.alloc(H.total);
    if (r->host_off == SIZE_MAX) return AMC_E_AGAIN;        // staging full: back-pressure
    if (!ses.known) {
        // first request: the session's table of status sets lives in the pool,
        // every variable starting as {(V,I)} (Section 3.2)
        const size_t off = s->pool.alloc(align_up((size_t)req->n_vars, 256));
        if (off == SIZE_MAX) {
            s->host.free(r->host_off, H.total);
            return AMC_E_NOMEM;
        }
        if (cudaMemsetAsync(s->pool.ptr(off), (int)(1u << AMC_ST_VI), (size_t)req->n_vars, s->ctl) != cudaSuccess ||
            cudaStreamSynchronize(s->ctl) != cudaSuccess)
            return AMC_E_CUDA;
        ses.known = true;
        ses.n_vars = req->n_vars;
        ses.table_off = off;
    }
    uint8_t* h = s->host.ptr(r->host_off);
    r->ticket = s->next_ticket++;
    r->t_submit = now_s();
    lock.unlock();
    // stage the inputs in pinned memory outside the lock (the slot is reserved)
    if (r->n && !borrowed) {
        memcpy(h + H.ks, req->kind_side, (size_t)r->n);
        memcpy(h + H.var, req->var, 4 * (size_t)r->n);
    }
    lock.lock();
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    s->cv.notify_one();
    return AMC_OK;
}

int amc_serve_poll(amc_server* s, uint64_t ticket, int* done, amc_result* out)
{
    if (!s || !done) return AMC_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return AMC_E_INVALID;
    const Request& r = *it->second;
    *done = r.state == 2;
    if (*done && out) {
        out->error = r.error;
        out->first_fault = r.first_fault;
        out->n_items = r.n;
        out->status = s->host.ptr(r.host_off) + host_layout(r.n, r.src_ks != nullptr).out;
        out->t_submit = r.t_submit;
        out->t_admit = r.t_admit;
        out->t_done = r.t_done;
        out->is_mask = r.is_mask;
    }
    return AMC_OK;
}

int amc_serve_completed(amc_server* s, uint64_t* tickets, int32_t cap, int32_t* n)
{
    if (!s || !n || cap < 0 || (cap > 0 && !tickets)) return AMC_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    int32_t k = 0;
    while (k < cap && !s->finished.empty()) {
        tickets[k++] = s->finished.front();
        s->finished.pop_front();
    }
    *n = k;
    return AMC_OK;
}

int amc_serve_release(amc_server* s, uint64_t ticket)
{
    if (!s) return AMC_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->state != 2) return AMC_E_INVALID;
    s->host.free(it->second->host_off, it->second->host_bytes);
    s->reqs.erase(it);
    return AMC_OK;
}

int amc_session_export(amc_server* s, uint64_t session_id, uint8_t* host_status, int32_t n_vars)
{
    if (!s || !host_status) return AMC_E_INVALID;
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            auto it = s->sessions.find(session_id);
            if (it == s->sessions.end() || it->second.n_vars != n_vars) return AMC_E_INVALID;
            bool pending = it->second.busy;
            for (const auto& q : s->queue)
                if (q->session == session_id) pending = true;
            if (!pending) {
                return cudaMemcpy(host_status, s->pool.ptr(it->second.table_off), (size_t)n_vars,
                                  cudaMemcpyDeviceToHost) == cudaSuccess
                           ? AMC_OK
                           : AMC_E_CUDA;
            }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int amc_server_destroy(amc_server* s)
{
    if (!s) return AMC_E_INVALID;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_one();
    }
    s->worker.join();
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (auto& kv : s->reqs)
        if (kv.second->host_off != SIZE_MAX) s->host.free(kv.second->host_off, kv.second->host_bytes);
    if (s->ctl) cudaStreamDestroy(s->ctl);
    s->pool.release();
    s->host.release();
    delete s;
    return AMC_OK;
}

}  // extern "C"
