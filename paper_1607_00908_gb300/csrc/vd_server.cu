// Served form: frames from many simulations, continuous batching.
//
// A server owns one batch whose instances are the simulations; each
// simulation's labels, centroids and links stay resident on the device.
// Frames are submitted as they arrive (device pointers owned by the caller).
// vd_server_poll runs the scheduler: it retires finished steps (in order,
// via CUDA events) and, while fewer than two steps are in flight, admits the
// oldest waiting frame of every idle simulation (at most one frame per
// simulation per step, at most max_batch simulations, and only while the
// resident state plus the admitted frames fit the HBM budget) and enqueues
// one step for them with vd_batch_push_subset. Frames that arrive while a
// step runs join the next step, so the device always has work queued.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <vector>

#include "vd.h"

vd_status vd_batch_gather_counts_async(vd_batch* b, const int* h_sims, int n, int* d_scratch, int* h_pinned_out);
long long vd_batch_resident_bytes(const vd_batch* b);

namespace {

long long now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    long long ticket;
    const float* field;
    long long t_submit;
    long long bytes;
};

struct Step {
    cudaEvent_t done;
    std::vector<int> sims;
    std::vector<Pending> frames;
    int slot;   // index of the pinned count buffer
};

}  // namespace

struct vd_server {
    vd_batch* b = nullptr;
    int n = 0;
    int max_batch = 0;
    long long budget = 0;
    long long resident = 0;
    long long inflight_bytes = 0;
    long long next_ticket = 0;
    cudaStream_t s = 0;
    std::vector<vd_config> cfg;
    std::vector<std::deque<Pending>> q;
    std::vector<char> busy;
    std::deque<Step> flight;
    std::vector<cudaEvent_t> ev_free;
    long long steps = 0, frames_done = 0;
    // two count buffers (one per step in flight): device scratch + pinned host
    int* d_cnt[2] = {nullptr, nullptr};
    int* h_cnt[2] = {nullptr, nullptr};
    int slot_busy[2] = {0, 0};
};

extern "C" {

vd_status vd_server_create(const vd_config* sims, int32_t n_sims, int64_t hbm_budget_bytes, int32_t max_batch,
                           vd_server** out) {
    if (!sims || n_sims < 1 || !out || hbm_budget_bytes <= 0 || max_batch < 1) return VD_ERR_INVALID;
    vd_server* sv = new (std::nothrow) vd_server();
    if (!sv) return VD_ERR_OOM;
    vd_status r = vd_batch_create(sims, n_sims, &sv->b);
    if (r) {
        delete sv;
        return r;
    }
    // resident state of every simulation: the bytes the batch allocated
    sv->resident = vd_batch_resident_bytes(sv->b) + 2ll * (long long)sizeof(int) * 7 * n_sims;
    if (sv->resident > hbm_budget_bytes) {
        vd_batch_destroy(sv->b);
        delete sv;
        return VD_ERR_CAPACITY;
    }
    for (int k = 0; k < 2; ++k) {
        if (cudaMalloc(&sv->d_cnt[k], sizeof(int) * 7 * n_sims) != cudaSuccess ||
            cudaMallocHost(&sv->h_cnt[k], sizeof(int) * 6 * n_sims) != cudaSuccess) {
            vd_batch_destroy(sv->b);
            delete sv;
            return VD_ERR_OOM;
        }
    }
    sv->n = n_sims;
    sv->max_batch = max_batch;
    sv->budget = hbm_budget_bytes;
    sv->s = (cudaStream_t)sims[0].stream;
    sv->cfg.assign(sims, sims + n_sims);
    sv->q.resize(n_sims);
    sv->busy.assign(n_sims, 0);
    *out = sv;
    return VD_OK;
}

vd_status vd_server_submit(vd_server* sv, int32_t sim, const float* d_field, int64_t* ticket) {
    if (!sv || sim < 0 || sim >= sv->n || !d_field) return VD_ERR_INVALID;
    Pending p;
    p.ticket = sv->next_ticket++;
    p.field = d_field;
    p.t_submit = now_ns();
    p.bytes = 4ll * sv->cfg[sim].Lx * sv->cfg[sim].Ly;
    sv->q[sim].push_back(p);
    if (ticket) *ticket = p.ticket;
    return VD_OK;
}

static vd_status server_launch(vd_server* sv) {
    // idle simulations with a waiting frame, oldest head frame first
    std::vector<int> cand;
    for (int i = 0; i < sv->n; ++i)
        if (!sv->busy[i] && !sv->q[i].empty()) cand.push_back(i);
    if (cand.empty()) return VD_OK;
    std::sort(cand.begin(), cand.end(),
              [&](int a, int b) { return sv->q[a].front().t_submit < sv->q[b].front().t_submit; });
    Step st;
    std::vector<const float*> fields;
    for (int i : cand) {
        if ((int)st.sims.size() >= sv->max_batch) break;
        const Pending& p = sv->q[i].front();
        if (sv->resident + sv->inflight_bytes + p.bytes > sv->budget) break;   // admission by HBM budget
        sv->inflight_bytes += p.bytes;
        st.sims.push_back(i);
        st.frames.push_back(p);
        fields.push_back(p.field);
        sv->q[i].pop_front();
        sv->busy[i] = 1;
    }
    if (st.sims.empty()) return VD_OK;
    vd_status r = vd_batch_push_subset(sv->b, st.sims.data(), (int32_t)st.sims.size(), fields.data());
    if (r) return r;
    st.slot = sv->slot_busy[0] ? 1 : 0;
    sv->slot_busy[st.slot] = 1;
    r = vd_batch_gather_counts_async(sv->b, st.sims.data(), (int)st.sims.size(), sv->d_cnt[st.slot],
                                     sv->h_cnt[st.slot]);
    if (r) return r;
    if (sv->ev_free.empty()) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return VD_ERR_CUDA;
        sv->ev_free.push_back(e);
    }
    st.done = sv->ev_free.back();
    sv->ev_free.pop_back();
    if (cudaEventRecord(st.done, sv->s) != cudaSuccess) return VD_ERR_CUDA;
    sv->flight.push_back(std::move(st));
    sv->steps += 1;
    return VD_OK;
}

vd_status vd_server_poll(vd_server* sv, int32_t wait, vd_server_done* done, int32_t cap, int32_t* n_done) {
    if (!sv || (cap > 0 && !done)) return VD_ERR_INVALID;
    int nd = 0;
    vd_status r = VD_OK;
    for (;;) {
        // retire finished steps in launch order
        while (!sv->flight.empty()) {
            Step& st = sv->flight.front();
            const cudaError_t q = cudaEventQuery(st.done);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) return VD_ERR_CUDA;
            if (nd + (int)st.sims.size() > cap) break;   // caller's buffer is full: retire later
            const long long t = now_ns();
            const int* c = sv->h_cnt[st.slot];
            for (size_t k = 0; k < st.sims.size(); ++k) {
                vd_server_done& d = done[nd++];
                d.ticket = st.frames[k].ticket;
                d.sim = st.sims[k];
                d.t_submit_ns = st.frames[k].t_submit;
                d.t_done_ns = t;
                d.n_bubbles = c[6 * k + 0];
                d.n_edges = c[6 * k + 1];
                d.n_breaking = c[6 * k + 2];
                d.n_arising = c[6 * k + 3];
                d.status = c[6 * k + 5] ? ((c[6 * k + 5] & 16) ? VD_ERR_TIMEOUT : VD_ERR_CAPACITY) : VD_OK;
                sv->busy[st.sims[k]] = 0;
                sv->inflight_bytes -= st.frames[k].bytes;
            }
            sv->slot_busy[st.slot] = 0;
            sv->frames_done += (long long)st.sims.size();
            sv->ev_free.push_back(st.done);
            sv->flight.pop_front();
        }
        // keep up to two steps queued on the device
        while (sv->flight.size() < 2) {
            const size_t before = sv->flight.size();
            r = server_launch(sv);
            if (r || sv->flight.size() == before) break;
        }
        if (r) break;
        if (!wait || nd > 0 || sv->flight.empty()) break;
    }
    if (n_done) *n_done = nd;
    return r;
}

vd_status vd_server_get_changes(vd_server* sv, int32_t sim, vd_changes* out) {
    if (!sv || sim < 0 || sim >= sv->n) return VD_ERR_INVALID;
    if (sv->busy[sim]) return VD_ERR_STATE;   // a frame of this simulation is still in flight
    return vd_batch_get_changes(sv->b, sim, out);
}

vd_status vd_server_get_labels(vd_server* sv, int32_t sim, int32_t* out, int64_t cap, int64_t* n) {
    if (!sv || sim < 0 || sim >= sv->n) return VD_ERR_INVALID;
    if (sv->busy[sim]) return VD_ERR_STATE;
    return vd_batch_get_labels(sv->b, sim, out, cap, n);
}

vd_status vd_server_stats(vd_server* sv, int64_t* steps, int64_t* frames_done, int64_t* resident_bytes,
                          int64_t* queued) {
    if (!sv) return VD_ERR_INVALID;
    if (steps) *steps = sv->steps;
    if (frames_done) *frames_done = sv->frames_done;
    if (resident_bytes) *resident_bytes = sv->resident;
    if (queued) {
        long long qn = 0;
        for (auto& d : sv->q) qn += (long long)d.size();
        *queued = qn;
    }
    return VD_OK;
}

vd_status vd_server_destroy(vd_server* sv) {
    if (!sv) return VD_ERR_INVALID;
    cudaStreamSynchronize(sv->s);
    for (auto& st : sv->flight) cudaEventDestroy(st.done);
    for (cudaEvent_t e : sv->ev_free) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        cudaFree(sv->d_cnt[k]);
        cudaFreeHost(sv->h_cnt[k]);
    }
    vd_batch_destroy(sv->b);
    delete sv;
    return VD_OK;
}

}  // extern "C"
